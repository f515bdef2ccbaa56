/*
 * dem.h -- C ABI of the GB300 soft-sphere DEM library (libdem.so).
 *
 * The library advances a scene of frictional spheres with the discrete element
 * method of the Yade documentation (3rd ed.), chapter 2 "DEM formulation":
 * the bounding-volume collider (section 2.1.1), the sphere-sphere and
 * wall-sphere contact geometry with incremental shear transport
 * (section 2.1.3; ScGeom, Ig2_Sphere_Sphere_ScGeom, Ig2_Wall_Sphere_ScGeom), the
 * FrictPhys stiffnesses (section 2.1.2; Ip2_FrictMat_FrictMat_FrictPhys), the
 * Cundall-Strack linear elastic-frictional law (section 2.1.4;
 * Law2_ScGeom_FrictPhys_CundallStrack), per-body force/torque summation and the
 * damped leapfrog of NewtonIntegrator (section 2.1.5, eq. 2.9), in an open box
 * with axis-aligned walls or in a deformable periodic cell (section 2.1.6).
 * Every step runs in CUDA kernels on one GPU; there is no CPU fallback.
 *
 * General rules
 *  - Every array argument is a HOST pointer unless its name ends in _dev.  The
 *    caller owns every host array: the library copies in or out and keeps no
 *    pointer after the call returns.  The library owns all device memory of a
 *    scene and frees it in dem_scene_destroy.
 *  - Vectors are packed xyz triples (n*3 doubles, row-major); quaternions are
 *    (w, x, y, z); 3x3 matrices are row-major with the periodic cell's base
 *    vectors in the COLUMNS (Cell.hSize).
 *  - Body ids are 0..n-1 in insertion order (section 1.1.2 "Bodies").  Arrays
 *    in and out of the library are in id order.
 *  - A scene is not thread-safe: drive one scene from one host thread.
 *    Different scenes may run concurrently on different streams.
 *  - Every call returns a dem_status; on error, dem_last_error(scene) returns a
 *    one-line message (valid until the next call on that scene).  Errors never
 *    leave the scene half-updated except where noted (DEM_ERR_CUDA,
 *    DEM_ERR_TIMEOUT: the scene is then unusable and should be destroyed).
 *  - Host waits are bounded (DEM_TIMEOUT_S environment variable, default 120
 *    seconds): a wait that expires returns DEM_ERR_TIMEOUT.
 */
#ifndef GB300_DEM_H
#define GB300_DEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dem_scene dem_scene; /* opaque, library-owned */

typedef enum dem_status {
    DEM_OK = 0,
    DEM_ERR_INVALID_ARG = 1,  /* bad argument (null pointer, negative size, unknown material) */
    DEM_ERR_OUT_OF_RANGE = 2, /* body id out of range (section 1.1.2, O.bodies[id]) */
    DEM_ERR_OOM = 3,          /* device or host allocation failed */
    DEM_ERR_CAPACITY = 4,     /* a fixed limit was exceeded (cell shift, cell count) */
    DEM_ERR_NONFINITE = 5,    /* NaN/Inf in an input or a body state during stepping */
    DEM_ERR_GEOMETRY = 6,     /* a sphere spans more than half the periodic cell (2.1.6) */
    DEM_ERR_TIMEOUT = 7,      /* a bounded host wait expired */
    DEM_ERR_CUDA = 8,         /* a CUDA runtime call failed */
    DEM_ERR_STATE = 9,        /* call not valid in the scene's state (e.g. no dt, lost history) */
    DEM_ERR_UNSUPPORTED = 10  /* valid request this version does not implement */
} dem_status;

enum { DEM_FP64 = 0, DEM_MIXED = 1 };

/* Scene description (POD).  Initialise with dem_scene_desc_init, then edit. */
typedef struct dem_scene_desc {
    int periodic;            /* 1: periodic cell cell_h (section 2.1.6); 0: open space */
    double cell_h[9];        /* periodic cell, base vectors in columns (row-major 3x3):
                                any parallelepiped with a positive diagonal and a
                                positive determinant; off-diagonal entries shear it */
    double box_lo[3];        /* walls: lower corner of the box */
    double box_hi[3];        /* walls: upper corner of the box */
    int wall_mask;           /* bit (2*axis + side): infinite wall at box_lo[axis] (side 0)
                                or box_hi[axis] (side 1), normal along axis, both senses;
                                ignored in periodic scenes (Wall shape, utils.wall) */
    double gravity[3];       /* NewtonIntegrator.gravity [m/s^2] */
    double damping;          /* NewtonIntegrator.damping, eq. 2.9 (default 0.2) */
    double dt;               /* time step; <= 0: 0.5 * PWaveTimeStep at the first step */
    double verlet_dist;      /* collider sweep margin dL (section 2.1.1, "Verlet distance"):
                                > 0 absolute; < 0 fraction of the smallest radius
                                (default -0.5, InsertionSortCollider.verletDist) */
    int precision;           /* DEM_FP64: every operation in double precision.
                                DEM_MIXED: contact geometry and law in FP32 on FP32 offsets
                                from each body's FP64 position at the last collider run
                                (per-row FP32 reference branch vectors); the shear-force
                                history and its rotation into the new contact frame, the
                                velocity/position accumulation and the kinetic-energy and
                                unbalanced-force reductions stay FP64. */
    long long capacity_bodies;   /* initial device capacity hint (0: grow on demand) */
    long long capacity_contacts; /* initial contact-table rows hint (0: grow on demand) */
    void *cuda_stream;       /* cudaStream_t to run on; NULL: the scene creates its own */
    int device;              /* CUDA device ordinal; < 0: the current device */
} dem_scene_desc;

/* Statistics of the current state (utils module reference: kineticEnergy,
 * unbalancedForce, avgNumInteractions, porosity, getStress). */
typedef struct dem_stats {
    long long iter;          /* steps taken (O.iter) */
    double time;             /* simulated time (O.time) */
    double dt;
    long long n_bodies;
    long long n_contacts;    /* real sphere-sphere contacts */
    long long n_wall_contacts;
    long long n_candidates;  /* rows of the contact table (potential interactions) */
    long long n_rebuilds;    /* collider runs */
    double kinetic_energy;   /* sum 1/2 (m v^2 + I w^2) */
    double unbalanced_force; /* mean |contact force on body| / mean |contact force| */
    double coordination;     /* Z = 2 C / N (sphere-sphere contacts) */
    double packing_fraction; /* sum of sphere volumes / cell (or box) volume */
    double stress[9];        /* Love-Weber (1/V) sum f l, compression negative */
} dem_stats;

/* Per-phase device time of dem_step, measured with CUDA events recorded on the
 * scene's stream around every launch while timing is enabled (Yade's per-engine
 * execTime / execCount, section 3.1.6 "Timing").  Times in milliseconds. */
typedef struct dem_timing {
    double contact_ms;            /* fused geometry + law kernel */
    double integrate_ms;          /* gather + integrator kernel */
    double cell_ms;               /* cell / clock advance */
    double collider_ms;           /* collider runs (all of their kernels and copies) */
    long long contact_launches;   /* counted per completed step (launches skipped after */
    long long integrate_launches; /* a collider request are timed but not counted)      */
    long long cell_launches;
    long long collider_runs;
    long long rows_processed;     /* sum over counted contact launches of table rows */
    long long kernel_launches;    /* every kernel this scene launched (timing on or off) */
} dem_timing;

/* Fill *desc with the defaults listed above.  Never fails. */
void dem_scene_desc_init(dem_scene_desc *desc);

/* Create an empty scene on the GPU.  desc is copied.  On success *out is a new
 * handle (free it with dem_scene_destroy).  Errors: INVALID_ARG (null, a periodic cell
 * with a non-positive diagonal entry or determinant, negative damping), CUDA, OOM. */
dem_status dem_scene_create(const dem_scene_desc *desc, dem_scene **out);

/* Release every resource of the scene (waits for its work to finish). NULL is a no-op. */
void dem_scene_destroy(dem_scene *scene);

/* FrictMat (Material / ElastMat / FrictMat class reference): density [kg/m^3],
 * young [Pa], poisson = ks/kn ratio, friction angle [rad] in [0, pi/2).
 * mat_id in [0, 4095].  Must precede dem_add_spheres that use it: mass and inertia
 * are fixed at insertion (utils.sphere).  Errors: INVALID_ARG. */
dem_status dem_set_material(dem_scene *scene, int mat_id, double density, double young,
                            double poisson, double friction_angle);

/* Append n spheres (utils.sphere): pos n*3, radius n (> 0), mat_id n (NULL: all 0),
 * vel/angvel n*3 (NULL: zero), fixed n (NULL: none; a fixed body keeps its velocities
 * and is not moved by forces).  Mass = density * 4/3 pi r^3, inertia = 2/5 m r^2.
 * *first_id (nullable) receives the id of the first new body.  Errors: INVALID_ARG,
 * NONFINITE, OOM, CUDA. */
dem_status dem_add_spheres(dem_scene *scene, long long n, const double *pos,
                           const double *radius, const int *mat_id, const double *vel,
                           const double *angvel, const unsigned char *fixed,
                           long long *first_id);

/* Time step (O.dt).  dt > 0.  dem_get_dt returns the step in use (computing the
 * default 0.5 * PWaveTimeStep if none was set and bodies exist). */
dem_status dem_set_dt(dem_scene *scene, double dt);
dem_status dem_get_dt(dem_scene *scene, double *dt);

/* Cell.velGrad for a periodic scene; like Cell.velGrad assignment the value takes
 * effect at the next step.  Any 3x3 (off-diagonal entries shear the cell; homoDeform = 2
 * moves every body with the full field).  Errors: INVALID_ARG, STATE (aperiodic). */
dem_status dem_set_cell_velgrad(dem_scene *scene, const double velgrad[9]);

/* Stress-controlled periodic cell (PeriTriaxController: goal, stressMask,
 * maxStrainRate, growDamping, globUpdate).  Every glob_update steps the diagonal
 * velocity gradient of each axis a is set, effective from the next step:
 *   stress_mask bit a set: grad(v)_aa = clamp((1 - grow_damping)(goal[a] - s_aa) /
 *     (K_a dt glob_update), +-max_rate[a]), with s the Love-Weber stress of that
 *     step's contacts (compression negative, Pa) and K_a = (1/V) sum kn (l n_a)^2;
 *   bit clear: grad(v)_aa = goal[a] (a strain rate, 1/s).
 * The text names these attributes but prints no update formula; this is the
 * formula both the library and its test oracle use.  The sums are FP64 in an FP64
 * scene; in a DEM_MIXED scene each contact's products are formed from its FP32
 * operands in FP32 and summed in FP32 over runs of 8 contacts, the runs in FP64
 * (relative error of a run at most 11 x 2^-23 of its terms' magnitudes).  Errors:
 * STATE (aperiodic), INVALID_ARG. */
dem_status dem_set_triax(dem_scene *scene, const double goal[3], int stress_mask,
                         const double max_rate[3], double grow_damping, int glob_update);

/* Peri3dController (class reference; the periodic-cell controllers named in section
 * 2.1.6) on a periodic scene without sub-scenes: the six components of the cell's
 * engineering stress and strain, in the order xx, yy, zz, yz, zx, xy (shear strains
 * are twice the tensor entries), each prescribed as a stress (stress_mask bit i set,
 * Pa, compression negative) or as a strain, along a time function of the progress
 * k / n_steps.  At the end of every step k the controller reads the Love-Weber stress
 * of that step's contacts (symmetrised, in the cell they were computed in) and the
 * strain U (P - I) U^T of Cell.trsf = H H0^-1 trsf0 = U P (polar decomposition; H0
 * the cell now), sets each strain component's rate to reach its path value at k + 1
 * and changes each stress component's rate by -+ mod x (largest current rate) when
 * the stress error extrapolated one step (2 e_k - e_(k-1)) is positive / negative
 * (the first update instead solves an isotropic elastic estimate with young_est,
 * poisson_est); rates are clamped to +-max_strain_rate and realised exactly by
 * grad v = (T+ T^-1 - I) / dt with T+ = U (P + U^T dt E U), assigned like
 * Cell.velGrad (from the next step).  It stops updating after n_steps or when a strain
 * component reaches max_strain; the last gradient stays in effect.  Readings: the
 * text gives the predictor and the rotation handling but not the first-step system,
 * the strain measure or the end; those are this library's.
 *   goal      HOST 6 doubles
 *   npath     HOST 6 ints (nullable: every path linear from 0 to the goal); npath[i]
 *             = 0 keeps the linear path of component i, else 1..16 couples
 *   path      HOST 6 x 16 x 2 doubles (t, v): times increasing from a positive first
 *             one; the last couple stands for (n_steps, goal) and scales the others
 *             (xxPath ... xyPath)
 *   trsf0     HOST 9 doubles (nullable: identity), Cell.trsf when the controller starts
 * Replaces the stress servo of dem_set_triax (and that call replaces this one).
 * Errors: STATE (aperiodic), UNSUPPORTED (sub-scenes), INVALID_ARG. */
dem_status dem_set_peri3d(dem_scene *scene, const double goal[6], int stress_mask,
                          long long n_steps, double mod, double max_strain_rate, double young_est,
                          double poisson_est, double max_strain, const int *npath,
                          const double *path, const double *trsf0);

/* The controller's last stress, strain and strain-rate vectors (HOST 6 doubles each,
 * nullable) and whether it has finished (done, nullable).  Errors: STATE (none set). */
dem_status dem_get_peri3d(dem_scene *scene, double *stress, double *strain, double *rate,
                          int *done);

/* Advance nsteps time steps (O.run(nsteps, wait=True)).  Blocks until done.
 * Errors: STATE (no bodies' dt), NONFINITE (a body state became NaN/Inf),
 * GEOMETRY, CAPACITY, OOM, TIMEOUT, CUDA.  On NONFINITE the scene stops at the
 * failing step. */
dem_status dem_step(dem_scene *scene, long long nsteps);

/* Copy the state out in id order.  pos/vel/angvel/force/torque n*3, ori n*4; each
 * nullable.  force/torque are the contact forces and torques of the last step
 * (O.forces.f / O.forces.t: gravity excluded). */
dem_status dem_get_state(dem_scene *scene, double *pos, double *vel, double *angvel, double *ori,
                         double *force, double *torque);

/* Overwrite body states (id order, each nullable).  Contact histories are kept and
 * re-matched at the next step; the collider re-runs. */
dem_status dem_set_state(dem_scene *scene, const double *pos, const double *vel,
                         const double *angvel, const double *ori);

/* Periodic cell state: H (hSize), velGrad in effect, previous velGrad and previous H
 * (each nullable).  Errors: STATE (aperiodic). */
dem_status dem_get_cell(dem_scene *scene, double *H, double *velgrad, double *prev_velgrad,
                        double *prev_H);
dem_status dem_set_cell(dem_scene *scene, const double *H, const double *velgrad,
                        const double *prev_velgrad, const double *prev_H);

/* utils.flipCell (section 2.1.6 "Collision detection in periodic cell", fig. 6) on
 * sub-scene `sub` (0 for a scene without sub-scenes).  The corners of the cell
 * repeated in space form a lattice that another cell H' = H M spans as well (M an
 * integer matrix with det M = 1); the flip replaces H by H M, keeps every body where
 * it is and every interaction on the same image (its cell shift c becomes M^-1 c),
 * and re-initialises the collider at the next step.  Flipping a sheared cell back
 * toward a right parallelepiped keeps the grid's cells from thinning as the shear
 * grows, so simple shear can go on without bound.
 *   flip     HOST 9 ints, row-major K with M = I + K, or NULL: the automatic
 *            reduction - one pass over the column pairs (i, j) in the order (1,2)
 *            (0,2) (0,1) (1,0) (2,0) (2,1), each replacing column j of the cell by
 *            column j - k column i with k = round(H_ij / H_ii) when k != 0 and H_jj
 *            stays positive (for a cell sheared in its upper triangle this leaves
 *            |H_ij| <= H_ii / 2)
 *   applied  HOST 9 ints (nullable): receives the K that was applied (zero: none)
 * Errors: INVALID_ARG (no such sub-scene, det(I + K) != 1, entries of K beyond
 * +-1000, a flipped cell with a non-positive diagonal), STATE (aperiodic),
 * GEOMETRY (some shift M^-1 c beyond +-511; nothing is changed), CUDA. */
dem_status dem_flip_cell(dem_scene *scene, int sub, const int *flip, int *applied);

/* O.iter and O.time. */
dem_status dem_get_clock(dem_scene *scene, long long *iter, double *time);
dem_status dem_set_clock(dem_scene *scene, long long iter, double time);

/* Number of real contacts (sphere-sphere plus sphere-wall) after the last step. */
dem_status dem_count_contacts(dem_scene *scene, long long *count);

/* Real interactions after the last step (O.interactions, which skips potential
 * ones), canonical order: sorted by (id1, id2), id1 < id2; a wall contact has
 * id1 = -(wall + 1) (wall = 2*axis + side) and sorts first.  Per row:
 * cell_dist 3 ints (Interaction.cellDist, applied to id2), normal_force and
 * shear_force 3 doubles each (FrictPhys normalForce / shearForce: acting on id2),
 * normal 3 (ScGeom.normal, from id1 to id2), contact_point 3 (x1 + (r1 - pen/2) n at
 * the current positions), phys 3 (kn, ks, tan(phi)), pen 1 (penetrationDepth).
 * Writes min(count, cap) rows; *count receives the total.  Output arrays nullable. */
dem_status dem_get_contacts(dem_scene *scene, long long cap, long long *count, int *id1,
                            int *id2, int *cell_dist, double *normal_force,
                            double *shear_force, double *normal, double *contact_point,
                            double *phys, double *pen);

/* Replace the contact history (checkpoint/resume): n rows in the canonical order of
 * dem_get_contacts, each with cell_dist (NULL: zero), the shear force on id2, the
 * normal of the last step and phys = (kn, ks, tan(phi)).  Rows whose pair is not in
 * contact at the next step are dropped there.  Errors: INVALID_ARG, OUT_OF_RANGE. */
dem_status dem_set_contacts(dem_scene *scene, long long n, const int *id1, const int *id2,
                            const int *cell_dist, const double *shear_force,
                            const double *normal_prev, const double *phys);

/* Statistics of the current state. */
dem_status dem_get_stats(dem_scene *scene, dem_stats *out);

/* Enable (1) or disable (0) per-phase timing; either call resets the counters
 * except kernel_launches.  Timing adds two event records per launch. */
dem_status dem_set_timing(dem_scene *scene, int enable);
dem_status dem_get_timing(dem_scene *scene, dem_timing *out);

/* ---- Sub-scenes: many independent scenes advanced by the same launches.
 *
 * A scene holds one or more sub-scenes.  Sub-scene 0 is the one its descriptor
 * defines (every single-scene call above acts on it); dem_add_subscene adds more,
 * each with its own periodic cell or box and walls, wall material, gravity,
 * damping, time step (so its own clock) and sweep margin, sharing the material
 * table, the precision and the launch shapes.  Bodies of different sub-scenes
 * never interact: the collider builds one grid per sub-scene.  One dem_step(n)
 * advances every sub-scene by n of its own steps with one launch per kernel for
 * all of them.  The paper has no counterpart (Yade runs one scene per process);
 * this is how the library batches parameter sweeps on one GPU.
 *
 * Ids: the spheres of a sub-scene have consecutive ids [first_id, first_id + n)
 * in the scene's id space, so dem_get_state / dem_get_contacts cover every
 * sub-scene at once.  Removing a sub-scene closes the gap at the next collider run
 * (the ids of the sub-scenes after it move down); dem_get_subscene reports the
 * current range.  The stress servo (dem_set_triax) runs only on a scene without
 * sub-scenes. */
typedef struct dem_subscene_desc {
    int periodic;            /* 1: periodic cell cell_h (as dem_scene_desc); 0: box */
    double cell_h[9];
    double box_lo[3], box_hi[3];   /* walls of an aperiodic sub-scene */
    int wall_mask;           /* bit 2*axis + side (side 0: low face), as dem_scene_desc */
    int wall_material;       /* material of the walls (set with dem_set_material) */
    double gravity[3];
    double damping;          /* eq. 2.9, in [0, 1) */
    double dt;               /* > 0: fixed; 0: 0.5 x p-wave step of its own spheres */
    double verlet_dist;      /* as dem_scene_desc */
} dem_subscene_desc;

/* Defaults: aperiodic, no walls, wall material 0, no gravity, damping 0.2, dt 0
 * (automatic), verlet_dist -0.5.  Never fails. */
void dem_subscene_desc_init(dem_subscene_desc *desc);

/* Add an empty sub-scene; *sub receives its index (a removed sub-scene's index may
 * be reused).  Errors: INVALID_ARG (bad descriptor, unknown wall material),
 * UNSUPPORTED (the scene runs the stress servo), OOM. */
dem_status dem_add_subscene(dem_scene *scene, const dem_subscene_desc *desc, int *sub);

/* dem_add_spheres for sub-scene `sub`.  Only the sub-scene that received the last
 * spheres (or an empty one) can grow: UNSUPPORTED otherwise. */
dem_status dem_add_spheres_to(dem_scene *scene, int sub, long long n, const double *pos,
                              const double *radius, const int *mat, const double *vel,
                              const double *angvel, const unsigned char *fixed,
                              long long *first_id);

/* Remove a sub-scene and its spheres (they leave the arrays at the next collider
 * run, which the next dem_step starts with).  INVALID_ARG for an unknown index. */
dem_status dem_remove_subscene(dem_scene *scene, int sub);

/* Current id range, clock and time step of a sub-scene (any pointer may be NULL). */
dem_status dem_get_subscene(dem_scene *scene, int sub, long long *first_id, long long *n,
                            long long *iter, double *time, double *dt);

/* dem_get_stats restricted to one sub-scene (packing fraction over its own cell or
 * box).  STATE when sub-scenes were added or removed since the last step. */
dem_status dem_get_subscene_stats(dem_scene *scene, int sub, dem_stats *out);

/* dem_set_cell_velgrad for a periodic sub-scene. */
dem_status dem_set_subscene_velgrad(dem_scene *scene, int sub, const double *velgrad);

/* Number of spheres in the scene's id space (all sub-scenes; spheres of a removed
 * sub-scene count until the next collider run closes their ids). */
dem_status dem_num_bodies(dem_scene *scene, long long *n);

/* dem_get_state for the ids [first_id, first_id + n) only (gathered on the device,
 * n records copied).  OUT_OF_RANGE when the range leaves [0, number of spheres). */
dem_status dem_get_state_range(dem_scene *scene, long long first_id, long long n, double *pos,
                               double *vel, double *angvel, double *ori);

/* ---- Serving: a continuous-batching request server over the sub-scenes.
 *
 * The paper has no counterpart (it runs one scene per process, section 1.1.2):
 * this is the serving pattern applied to the method's hot path, for parameter
 * sweeps of packings and loading paths submitted as independent requests.  A
 * request is one scene (a sub-scene descriptor, its materials, its spheres, an
 * optional velocity gradient of its periodic cell) and a step budget.  A worker
 * thread owns one device scene; requests wait in arrival order and are admitted
 * as sub-scenes while their estimated device footprint fits the budget:
 *     bodies x (bytes per body + rows per body x bytes per table row),
 * the rows per body measured on the device after every tick (never below
 * rows_per_body).  First come, first served: a request that does not fit blocks
 * the ones behind it, so none starves.  Every tick advances all resident scenes by
 * the same number of steps (the smallest remaining budget, at most tick_steps) in
 * one dem_step; finished scenes are read to the host and removed at the end of the
 * tick they finish in, and waiting requests are admitted before the next tick.
 * Scene state stays on the device between ticks.  Requests submitted while others
 * run join at the next tick, so their work overlaps on the GPU.
 *
 * Results: in DEM_FP64 a request's result is bitwise the same as the same scene
 * run alone with dem_scene_create / dem_step (rows are oriented by id and every
 * per-body sum runs in increasing partner id, so other sub-scenes and the times
 * of the collider runs change nothing).  In DEM_MIXED the FP32 offsets from the
 * positions at the last collider run depend on when the collider ran, so results
 * agree with the run alone to the mixed-precision tolerance, not bitwise.
 *
 * Threads: every dem_server_* call is thread-safe; the device work runs on the
 * server's own worker thread (and stream).  Times are seconds of a steady clock
 * since dem_server_create. */
typedef struct dem_server dem_server;   /* opaque, library-owned */

typedef struct dem_server_desc {
    int precision;              /* DEM_FP64 or DEM_MIXED (default) */
    long long budget_bytes;     /* device-memory budget of the resident requests;
                                   0: half of the device memory free at creation */
    long long tick_steps;       /* most steps between two admission points (default 200) */
    double rows_per_body;       /* initial estimate of table rows per body (default 8) */
    void *cuda_stream;          /* stream of the worker; NULL: the server creates one */
    int device;                 /* CUDA device; < 0: the caller's current device */
} dem_server_desc;

/* Request: the scene is copied at submission (the caller may free its arrays once
 * dem_server_submit returns). */
typedef struct dem_request {
    dem_subscene_desc scene;    /* cell or box, walls, gravity, damping, dt (0: 0.5 x
                                   p-wave step of its spheres), verlet_dist;
                                   scene.wall_material indexes `materials` */
    int n_materials;            /* 1 .. 64 */
    const double *materials;    /* n_materials x 4: density, Young's modulus, Poisson
                                   ratio (ks/kn), friction angle [rad] (dem_set_material) */
    long long n;                /* spheres, >= 1 */
    const double *pos;          /* n x 3 */
    const double *radius;       /* n */
    const int *mat_id;          /* n indices into materials; NULL: all 0 */
    const double *vel;          /* n x 3 or NULL */
    const double *angvel;       /* n x 3 or NULL */
    const double *velgrad;      /* 9 (row-major) for a periodic scene, or NULL */
    long long nsteps;           /* step budget, >= 1 */
    int keep_state;             /* 1: keep the final state for dem_server_result */
} dem_request;

/* Result of a finished request. */
typedef struct dem_request_result {
    long long ticket, n, nsteps;
    long long iter;             /* steps taken (== nsteps) */
    double time, dt;            /* simulated time and step of the scene */
    double t_submit, t_admit, t_done;
    double latency;             /* t_done - t_submit */
    dem_stats stats;            /* dem_get_subscene_stats at the end */
} dem_request_result;

typedef struct dem_server_summary {
    long long submitted, completed, failed, waiting, resident;
    long long resident_bodies, max_resident;
    long long ticks, scene_steps, body_steps;
    long long budget_bytes;        /* the budget in force */
    long long resident_bytes_est;  /* footprint estimate of the resident requests */
    long long device_bytes;        /* largest device memory the scene has held */
    double rows_per_body;          /* the estimate admission uses now */
    double wall_s;                 /* since creation */
    double busy_s;                 /* inside dem_step */
    double latency_p50, latency_p99, latency_max, latency_mean;   /* finished requests */
    double concurrency_mean;       /* resident requests per tick */
    /* ticks by the number r of resident requests: [0] r = 1, [b] for b = 1..6
     * 2^(b-1) < r <= 2^b, [7] r > 64 */
    long long concurrency_hist[8];
} dem_server_summary;

/* Defaults of dem_server_desc (above).  Never fails. */
void dem_server_desc_init(dem_server_desc *desc);

/* Start a server (creates its device scene and worker thread; the caller's current
 * device is left as it was).  Errors: INVALID_ARG, CUDA, OOM. */
dem_status dem_server_create(const dem_server_desc *desc, dem_server **out);

/* Stop the worker after its current tick and free everything; requests not yet
 * finished are dropped. */
void dem_server_destroy(dem_server *server);

/* Zero *req and give req->scene the sub-scene defaults.  Never fails. */
void dem_request_init(dem_request *req);

/* Queue a request; *ticket identifies it.  Never waits for the GPU.  Errors:
 * INVALID_ARG (n < 1, nsteps < 1, missing arrays, material indices out of range),
 * CAPACITY (its footprint alone exceeds the budget), or the error that stopped a
 * failed server.  Scene errors found at admission (e.g. a sphere too large for its
 * periodic cell) fail that request only. */
dem_status dem_server_submit(dem_server *server, const dem_request *req, long long *ticket);

/* *state: 0 waiting, 1 resident, 2 done, 3 failed.  INVALID_ARG: unknown ticket. */
dem_status dem_server_poll(dem_server *server, long long ticket, int *state);

/* Block until the request is finished or timeout_s seconds have passed: OK (done),
 * TIMEOUT, the request's own error if it failed, INVALID_ARG (unknown ticket). */
dem_status dem_server_wait(dem_server *server, long long ticket, double timeout_s);

/* Copy a finished request's result: *info (nullable) and, if it was submitted with
 * keep_state, its final state in id order (each array nullable: n x 3, ori n x 4).
 * STATE: not finished; INVALID_ARG: unknown ticket, or state asked without
 * keep_state; the request's error if it failed. */
dem_status dem_server_result(dem_server *server, long long ticket, dem_request_result *info,
                             double *pos, double *vel, double *angvel, double *ori);

/* Forget a finished request (its result memory is freed).  STATE: not finished. */
dem_status dem_server_release(dem_server *server, long long ticket);

/* Counters, footprint and latency percentiles (linear interpolation between order
 * statistics) of the finished requests. */
dem_status dem_server_stats(dem_server *server, dem_server_summary *out);

/* Message of the last error of a dem_server_* call on this server (NULL server: of
 * a failed dem_server_create in this thread). */
const char *dem_server_last_error(dem_server *server);

/* Launch shapes of the step kernels.  No shape changes a result: every table row
 * and every body is computed by one thread with the same arithmetic whatever the
 * shape, so two scenes that differ only in their tuning follow bit-identical
 * trajectories.  (The paper's counterpart is the choice of OpenMP thread count,
 * section 3.1.6; this library exposes the GPU launch geometry instead.)
 *   contact_block          threads per block of the contact kernel: 128 or 256
 *   contact_blocks_per_sm  blocks per SM of the contact kernel's persistent grid,
 *                          1..64 (each warp walks rows/(SMs*blocks*block/32) rows)
 *   integrate_block        threads per block of the integrator: 128, 256 or 512
 *   degree_order           1: integrate the bodies of each run of 1024 slots in
 *                          decreasing order of incident contact rows (lanes of a warp
 *                          get similar row counts, a block's bodies stay neighbours);
 *                          0: in slot order
 *   step_graphs            1: a batch of steps is captured once as a CUDA graph and
 *                          replayed (one launch per batch; the kernels then read
 *                          tables and bodies through a device-resident descriptor, so
 *                          a capture stays valid across collider runs until the body
 *                          count, a table capacity, a launch shape or the sub-scene
 *                          count changes); 0: every kernel launched one by one, with
 *                          the arrays as launch parameters (fewer registers);
 *                          -1: graphs below 262,144 bodies, where launch overhead
 *                          matters.  Batches with per-kernel timing, the stress servo
 *                          or the time stepper are never captured.
 * Defaults: 256, 8, 256, 1, -1. */
typedef struct dem_tuning {
    int contact_block;
    int contact_blocks_per_sm;
    int integrate_block;
    int degree_order;
    int step_graphs;
} dem_tuning;

/* Set the launch shapes (INVALID_ARG outside the ranges above) or read them. */
dem_status dem_set_tuning(dem_scene *scene, const dem_tuning *tuning);
dem_status dem_get_tuning(const dem_scene *scene, dem_tuning *tuning);

/* Pick the launch shapes by timing the scene's own steps: six contact-kernel
 * shapes (block 128/256 x 4/8/16 blocks of 256 threads per SM), each timed twice in
 * two passes and taken per table row processed (a scene that gains contacts during
 * the trials does not favour the shapes tried first), then five more integrator
 * shapes (block 128/256/512 x body order) with the best contact shape (step_graphs is
 * left as set: per-kernel timing runs without graphs); each trial is one untimed
 * step plus steps_per_trial timed steps (CUDA events around each kernel; collider
 * runs excluded).  The trial steps are real steps: the scene advances by
 * 17 * (steps_per_trial + 1) steps, along the trajectory
 * any fixed shape gives.  The best shape is applied and, if chosen is non-null,
 * written there.  Errors: INVALID_ARG (steps_per_trial < 1), those of dem_step. */
dem_status dem_autotune(dem_scene *scene, long long steps_per_trial, dem_tuning *chosen);

/* Contact law of a sub-scene (0 for a plain scene), chosen before its first step
 * (STATE afterwards, INVALID_ARG for an unknown law):
 *   DEM_LAW_LINEAR          Ip2_FrictMat_FrictMat_FrictPhys + Law2_ScGeom_FrictPhys_
 *                           CundallStrack (the default): Fn = kn pen
 *   DEM_LAW_HERTZ_MINDLIN   Ip2_FrictMat_FrictMat_MindlinPhys + Law2_ScGeom_MindlinPhys_
 *                           Mindlin (class references): Fn = kno pen^3/2 with
 *                           kno = 4/3 E* sqrt(R*), shear stiffness kso pen^1/2 with
 *                           kso = 8 sqrt(R*) / ((2-nu1)/G1 + (2-nu2)/G2) (2 sqrt(4R) G /
 *                           (2 - nu) for equal materials, as the text writes),
 *                           1/E* = sum (1 - nu^2)/E, R* = r1 r2 / (r1 + r2) (a wall: r),
 *                           G = E / (2 (1 + nu)), the material's poisson being the true
 *                           Poisson ratio; the same shear transport and Coulomb cap; no
 *                           viscous damping, adhesion or rolling moments.
 * dem_get_contacts then reports (kno, kso, tan phi) in phys. */
enum { DEM_LAW_LINEAR = 0, DEM_LAW_HERTZ_MINDLIN = 1 };
dem_status dem_set_law(dem_scene *scene, int sub, int law);

/* GlobalStiffnessTimeStepper (section 2.1.5 "Stability considerations", eq. 2.12 -
 * 2.14; class reference) for sub-scene `sub` (0 for a plain scene).  On every step
 * whose count is a multiple of `interval`, after the contact pass and before the
 * integration (the engine order of the text's scripts, so the new dt already
 * integrates that step), dt becomes `safety` times the smallest sqrt(2) sqrt(m / K)
 * over the free spheres and their six degrees of freedom taken as uncoupled:
 * translational K_ii = sum (kn - ks) n_i^2 + ks (eq. 2.14) and rotational
 * K_ii = sum ks d^2 (1 - n_i^2) over the sphere's contacts (d = r - pen/2, the arm of
 * the shear spring).  With no contact dt = default_dt, or (default_dt <= 0) safety x
 * the p-wave step of the sub-scene's spheres; max_dt > 0 caps it.  Density scaling:
 * dem_set_density_scaling.  Errors: INVALID_ARG (safety outside (0, 1], interval < 1). */
dem_status dem_set_timestepper(dem_scene *scene, int sub, double safety, int interval,
                               double default_dt, double max_dt);

/* Density scaling (NewtonIntegrator.densityScaling with GlobalStiffnessTimeStepper
 * targetDt, class references; the stability discussion of section 2.1.5) for
 * sub-scene `sub`, which must run the time stepper.  On each stepper update every
 * free sphere with contacts gets an inertia factor f = (target_dt / (safety t_b))^2,
 * t_b its own critical step of eq. 2.12 (true mass and inertia, the six degrees of
 * freedom of dem_set_timestepper), and the step becomes target_dt: every sphere then
 * sits at the same stability margin, which speeds up quasi-static runs at the cost of
 * realistic dynamics.  Mass and moment of inertia are both multiplied by f in the
 * equations of motion; forces are not changed (the weight stays the true m g), so a
 * static equilibrium does not depend on target_dt.  A sphere without contacts keeps
 * its last factor (1 at first).  enable = 0 switches it off and restores f = 1.
 * Errors: INVALID_ARG (no such sub-scene, target_dt not finite and > 0), STATE (no
 * time stepper on the sub-scene). */
dem_status dem_set_density_scaling(dem_scene *scene, int sub, int enable, double target_dt);

/* The inertia factor f of every sphere, by id (HOST n doubles, n = dem_num_bodies). */
dem_status dem_get_density_scaling(dem_scene *scene, double *f);

/* Micromechanics of the contacts of the last completed step (utils reference of
 * the text), over the whole scene (sub = -1, volume of sub-scene 0) or one
 * sub-scene:
 *   fabric         fabricTensor: (1/n_c) sum n (x) n over sphere-sphere contacts
 *   normal_stress  normalShearStressTensors, normal part: -(1/V) sum l N n (x) n
 *   shear_stress   shear part: -(1/V) sum l n (x) Fs
 * n = contact normal, l = current centroid distance, N = normal force (> 0 in
 * compression), Fs = shear force on body 2, V = cell (periodic) or box volume;
 * compression negative, so normal_stress + transpose(shear_stress) equals the
 * stress of dem_get_stats.  Row-major 3x3 HOST outputs (any may be NULL); zeros
 * before the first step.  Sums in a fixed order: reproducible bit for bit. */
dem_status dem_get_micro(dem_scene *scene, int sub, double *fabric, double *normal_stress,
                         double *shear_stress, long long *n_contacts);

/* bodyStressTensors: per sphere (1/V_b) sum x (x) f over its contacts (spheres and
 * walls), x the contact point relative to its centre, f the force on it, V_b the
 * sphere volume.  out: HOST n_bodies * 9 doubles in id order (row-major). */
dem_status dem_get_body_stress(dem_scene *scene, double *out);

/* Collision detection on a bare configuration (section 2.1.1, both passes: the
 * grid's bounding-volume filter, then the exact sphere test): every pair
 * i < j of the caller's indices with |x_j + H c - x_i| < (r_i + r_j) + margin,
 * c the cell shift of j (periodic cells: H = cell_h, diagonal; the shift of the
 * nearest image).  The exact test is evaluated in double precision with
 * round-to-nearest operations in the order written, so the set is exactly the
 * one this definition gives.
 *   pos_dev     DEVICE n*3 doubles; radius_dev DEVICE n doubles (> 0, finite)
 *   cell_h      HOST 9 doubles (read only when periodic)
 *   id1_dev, id2_dev  DEVICE cap ints; cell_dist_dev DEVICE cap*3 ints (nullable)
 *   count       HOST: receives the number of pairs; when it exceeds cap only the
 *               first cap rows are written (call again with a larger cap).
 * Rows come in a fixed order (grouped by the grid order of the sphere that
 * found them), the same on every call.  Scratch memory is allocated on
 * cuda_stream (NULL: the default stream) and freed before returning; the call
 * waits for its work.  Errors (reported by dem_last_error(NULL)): INVALID_ARG,
 * NONFINITE, GEOMETRY (a sphere pair spans a third of the periodic cell), OOM,
 * TIMEOUT, CUDA. */
dem_status dem_find_pairs(const double *pos_dev, const double *radius_dev, long long n,
                          int periodic, const double *cell_h, double margin, long long cap,
                          int *id1_dev, int *id2_dev, int *cell_dist_dev, long long *count,
                          void *cuda_stream);

/* dem_find_pairs without any allocation.  The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory at the time of the
 * call -- for example a program whose device memory is already reserved by
 * another framework's memory pool, or a latency-sensitive loop that must not
 * make the allocator's calls (which can synchronize the device).
 * Same arguments, results and errors as dem_find_pairs, with these limits:
 *   - at most 65,536 spheres (larger n: DEM_ERR_CAPACITY with a message naming
 *     dem_find_pairs) and at most 64 grid cells per axis;
 *   - its scratch is one fixed ~10 MB device array inside the library.  CUDA
 *     loads a library's device code lazily, so the array is reserved on a device
 *     by the first pair query there (this entry point or dem_find_pairs), and then
 *     held until the process exits.  A caller whose memory pool will take the
 *     rest of the device should make one call first, before the pool reserves
 *     memory: a call with n = 0 does only this set-up;
 *   - the first call on a device looks up that array's device address (a one-time
 *     set-up per device, cached): make that first call before any stream capture.
 *     cudaDeviceReset invalidates the cached address: do not call this entry point
 *     on a device after resetting it;
 *   - every call uses the same array, so calls whose work overlaps on the GPU
 *     (other threads, other streams) race and must be serialized by the caller;
 *     each call clears the parts that must start at zero;
 *   - the call waits for its work with a bounded poll (DEM_TIMEOUT_S, default
 *     120 s).  After DEM_ERR_TIMEOUT the call's kernels may still be running on
 *     cuda_stream and using the array: wait for that stream to drain (for
 *     example cudaStreamSynchronize) before the next call.
 * The caller still provides the input and output arrays. */
dem_status dem_find_pairs_noalloc(const double *pos_dev, const double *radius_dev, long long n,
                                  int periodic, const double *cell_h, double margin,
                                  long long cap, int *id1_dev, int *id2_dev, int *cell_dist_dev,
                                  long long *count, void *cuda_stream);

/* Measured FP64 throughput of this GPU in TFLOP/s: the denominator of the FP64
 * kernels' roofline.  The paper has no counterpart.  Each thread of a grid of
 * resident 256-thread blocks on every SM runs sixteen independent fused
 * multiply-add chains for `iters` iterations (rounded up to a multiple of 4; 2 flops
 * each); *tflops receives the
 * best rate of `repeats` timed launches after one warm-up launch (CUDA events on
 * cuda_stream, NULL: the default stream; a few bytes of scratch are allocated on it
 * and freed).  Waits are bounded (DEM_TIMEOUT_S).  Errors: INVALID_ARG (iters < 1,
 * repeats < 1, null tflops), TIMEOUT, CUDA (dem_last_error(NULL)). */
dem_status dem_measure_fp64_peak(long long iters, int repeats, void *cuda_stream,
                                 double *tflops);

/* Message of the last error on this scene ("" if none).  NULL scene: the last
 * error of a failed dem_scene_create or dem_find_pairs in this thread. */
const char *dem_last_error(const dem_scene *scene);

/* Library version string. */
const char *dem_version(void);

#ifdef __cplusplus
}
#endif
#endif
