/*
 * Plain FP64 CPU oracle of the soft-sphere DEM timestep (Yade documentation,
 * 3rd ed., chapter 2 "DEM formulation").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the package smoke check and the bench's CPU-baseline leg may
 * load or call it; the product path never does, and it shares no code, header,
 * helper or constant with the CUDA library.
 *
 * Conventions (all double precision, SI units):
 *   - bodies are spheres with ids 0..n-1 in insertion order;
 *   - a sphere-sphere contact is (id1 < id2, c) with c the integer cell shift
 *     applied to body id2 (Interaction.cellDist, section 2.1.6);
 *   - a sphere-wall contact has id1 = -(wall+1), wall = 2*axis + side;
 *   - normal n points from body 1 to body 2; forces are stored as acting on
 *     body 2 ("as sustained by particle #2", FrictPhys);
 *   - matrices are row-major 3x3; the periodic cell H holds base vectors in its
 *     columns (Cell.hSize).
 * Return codes: 0 ok, <0 error (-1 bad argument, -2 out of memory,
 * -3 geometry: sphere larger than half the cell, -4 unsupported).
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_scene orc_scene;

orc_scene *orc_create(int periodic, const double *H9, const double *box_lo, const double *box_hi,
                      int wall_mask, const double *gravity, double damping, double dt);
void orc_destroy(orc_scene *s);
int orc_set_material(orc_scene *s, int mat, double density, double young, double poisson,
                     double friction_angle);
long orc_add_spheres(orc_scene *s, long n, const double *pos, const double *radius,
                     const int *mat, const double *vel, const double *angvel,
                     const unsigned char *fixed);
int orc_set_dt(orc_scene *s, double dt);
int orc_set_velgrad(orc_scene *s, const double *L9);
int orc_step(orc_scene *s, long nsteps);
/* stress-controlled periodic cell (PeriTriaxController, reading R16 in dem_oracle.c) */
/* contact law: 0 linear Cundall-Strack (default), 1 Hertz-Mindlin (reading R18) */
int orc_set_law(orc_scene *s, int law);
/* GlobalStiffnessTimeStepper: safety coefficient, update interval (steps), defaultDt
 * (< 0: safety x p-wave step), maxDt (<= 0: none). */
/* density scaling (R22); f receives the per-body inertia factors (n doubles). */
int orc_set_density_scaling(orc_scene *s, int on, double target_dt);
void orc_get_density_scaling(const orc_scene *s, double *f);
/* Peri3dController (reading R23); path: [6][16][2] couples, npath[6] (nullable). */
int orc_set_peri3d(orc_scene *s, const double *goal, int stress_mask, long n_steps, double mod,
                   double max_strain_rate, double young_est, double poisson_est,
                   double max_strain, const int *npath, const double *path, const double *trsf0);
int orc_get_peri3d(const orc_scene *s, double *stress, double *strain, double *rate);
int orc_set_timestepper(orc_scene *s, double safety, int interval, double default_dt,
                        double max_dt);
int orc_set_triax(orc_scene *s, const double *goal3, int stress_mask, const double *max_rate3,
                  double grow_damping, int glob_update);

long orc_num_bodies(const orc_scene *s);
void orc_get_state(const orc_scene *s, double *pos, double *vel, double *angvel, double *ori,
                   double *force, double *torque);
int orc_set_state(orc_scene *s, const double *pos, const double *vel, const double *angvel,
                  const double *ori);
void orc_get_cell(const orc_scene *s, double *H9, double *velgrad9, double *prev_velgrad9,
                  double *prev_H9);
int orc_set_cell(orc_scene *s, const double *H9, const double *velgrad9,
                 const double *prev_velgrad9, const double *prev_H9);
/* utils.flipCell: H' = H (I + K), interactions keep their images (c' = (I + K)^-1 c).
 * K9 NULL: automatic reduction (reading R21).  applied (nullable) receives K. */
int orc_flip_cell(orc_scene *s, const int *K9, int *applied);
void orc_get_clock(const orc_scene *s, long *iter, double *time, double *dt);
int orc_set_clock(orc_scene *s, long iter, double time);

long orc_num_contacts(const orc_scene *s);
/* phys: kn, ks, tan(phi) per row; geom: pen per row.  Returns rows written. */
long orc_get_contacts(const orc_scene *s, long cap, int *id1, int *id2, int *c, double *fn,
                      double *fs, double *normal, double *cpoint, double *phys, double *pen);
/* history import: fs = shear force on body 2, nprev = normal of the last step. */
int orc_set_contacts(orc_scene *s, long n, const int *id1, const int *id2, const int *c,
                     const double *fs, const double *nprev, const double *phys);

/* kinTrans, kinRot, gravWork, nonviscDamp, plastDissip, elastPotential, total */
void orc_get_energy(const orc_scene *s, double *out7);
/* ke, unbalanced, Z, packing fraction, n_contacts(sphere-sphere), stress[9] */
void orc_get_stats(const orc_scene *s, double *out14);

double orc_sphere_pwave_dt(double radius, double density, double young);
double orc_pwave_dt(const orc_scene *s);

/* Pair searches on a bare configuration: all (i<j, c) with |x_j + H c - x_i| < r_i + r_j
 * + margin (aperiodic when periodic == 0).  Returns the count (may exceed cap; rows beyond
 * cap are not written), or <0 on error.  Rows sorted by (i, j). */
long orc_pairs_bruteforce(long n, const double *pos, const double *radius, int periodic,
                          const double *H9, double margin, long cap, int *i, int *j, int *c);
long orc_pairs_sweep(long n, const double *pos, const double *radius, int periodic,
                     const double *H9, double margin, long cap, int *i, int *j, int *c);
long orc_pairs_grid(long n, const double *pos, const double *radius, int periodic,
                    const double *H9, double margin, long cap, int *i, int *j, int *c);

#ifdef __cplusplus
}
#endif
#endif
