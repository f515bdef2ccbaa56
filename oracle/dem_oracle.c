/*
 * Plain FP64 CPU oracle of the soft-sphere DEM timestep.
 *
 * TEST INFRASTRUCTURE ONLY: this file checks the CUDA path and is never part of
 * the product.  Only the test suite, the package smoke check and the bench's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library.
 *
 * It follows the Yade documentation (3rd ed.), chapter 2 "DEM formulation",
 * step by step and in the text's order (simulation loop of section 1.1.2,
 * "Engines": ForceResetter -> collider -> InteractionLoop(Ig2, Ip2, Law2) ->
 * NewtonIntegrator), written the slow and obvious way:
 *
 *   - contact detection every step: candidates from a uniform cell list (cells
 *     as wide as the largest contact distance, the "grid algorithms" of
 *     section 2.1.1) followed by the exact sphere test; no Verlet distance is
 *     needed because the search runs every step.  A brute-force O(N^2) search
 *     and a sort-and-sweep along one axis (the "initial step" of the
 *     sweep-and-prune collider) check it;
 *   - interactions keyed by (id1, id2) in a sorted list carried from step to
 *     step (potential/real lifecycle, section 3.1.7 "Interactions");
 *   - Ig2_Sphere_Sphere_ScGeom: normal and contact point (eq. 2.7, 2.8),
 *     shear-force transport (section 2.1.3 "Shear deformation") with the
 *     ratchet-free relative velocity of the ScGeom class reference;
 *   - Ip2_FrictMat_FrictMat_FrictPhys (section 2.1.2 "Normal stiffness" and the
 *     class reference): series springs with l_i = 2 r_i;
 *   - Law2_ScGeom_FrictPhys_CundallStrack (section 2.1.4): Fn = kn*pen, trial
 *     shear force, Coulomb cap;
 *   - NewtonIntegrator (section 2.1.5): non-viscous damping (eq. 2.9),
 *     leapfrog for position and spherical rotation, orientation quaternion;
 *   - periodic cell (section 2.1.6 and Cell class reference): cellDist
 *     shifts, F+ = (I + grad(v) dt) F, homoDeform = 2 velocity terms.
 *
 * Readings where the text is silent, ambiguous or garbled (each one is listed
 * with its reason in the design notes of the repository):
 *   R1 real iff |x2 + H c - x1|^2 < (r1 + r2)^2 (strict; interactionDetectionFactor 1).
 *   R2 shear force stored as acting on body 2; increment Fs -= ks*dt*v12_perp.
 *   R3 v12 = ((r1+r2)/l)(v2 - v1) - (r2 w2 + r1 w1) x n (ScGeom class reference).
 *   R4 torques T_i = (C - x_i) x F_i, C = x1 + (r1 - pen/2) n (eq. 2.8).
 *   R5 both rotation increments of the shear transport use the previous shear
 *      force, as the equations of section 2.1.3 are written; the capped force
 *      (not the elastic displacement) is stored (FrictPhys "shear force after
 *      previous step").
 *   R6 a new contact starts with Fs = 0 and n_prev = n; the increment of the
 *      creation step is applied.
 *   R7 damping (eq. 2.9) applies to the total force including gravity
 *      (dampGravity = true) and, the same way, to torques; sgn(0) = 0.  In a
 *      periodic cell the velocity in eq. 2.9 is the fluctuation v - grad(v)_prev x.
 *   R8 image velocity of body 2 across the cell: v2 + grad(v)_prev H_prev c.
 *   R9 homoDeform = 2: v+ += (grad(v) - grad(v)_prev) x + dt grad(v) v-.
 *   R10 sphere-wall: n = +-e_axis from the wall to the sphere centre,
 *      pen = r - |x_a - w|, refR1 = refR2 = r (so kn = E r for equal E), l = 2r - pen,
 *      wall at rest; wall material = material 0.
 *   R11 fixed bodies keep their velocities (no force integration) and still move
 *      with them.
 *   R12 sphere inertia I = 2/5 m r^2, mass = density * 4/3 pi r^3 (utils.sphere).
 *   R16 PeriTriaxController (attributes only in the text: goal, stressMask,
 *      maxStrainRate, globUpdate, growDamping): every globUpdate steps, from the
 *      contacts of that step and the cell volume they were computed in,
 *      sigma_ii = (1/V) sum F_i (x1 - x2')_i (Love-Weber, compression negative) and
 *      K_i = (1/V) sum kn (l n_i)^2; a stress-controlled axis (stressMask bit i) gets
 *      grad(v)_ii = clamp((1 - growDamping)(goal_i - sigma_ii) / (K_i dt globUpdate),
 *      +-maxRate_i) -- the rate that closes (1 - growDamping) of the stress gap over
 *      the globUpdate steps it is held for
 *      (0 when K_i = 0 and the goal is not met: the rate bound applies), a
 *      strain-controlled axis grad(v)_ii = goal_i; the new gradient is assigned
 *      like Cell.velGrad (effective from the next step) and held in between.
 *   R22 density scaling (NewtonIntegrator.densityScaling, GlobalStiffnessTimeStepper
 *      targetDt; the text gives the purpose, equalising every body's critical step
 *      at targetDt, not the formula): on a stepper update a free body with contacts,
 *      critical step t_b of eq. 2.12 with its true mass and inertia, gets the factor
 *      f = (targetDt / (safety t_b))^2 on both; the step becomes targetDt.  Only the
 *      inertia is scaled: forces, weight m g included, are unchanged, so a static
 *      state does not depend on targetDt.  A body without contacts keeps its factor.
 */
#include "dem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_MAT 64

typedef struct {
    double density, young, poisson, friction;
    int set;
} orc_mat;

typedef struct {
    int id1, id2;          /* id1 < id2; id1 = -(wall+1) for a wall contact */
    int c[3];              /* cell shift applied to body id2 */
    double kn, ks, tanphi; /* FrictPhys, set at creation (Ip2) */
    double fs[3];          /* shear force on body 2 (history) */
    double nprev[3];       /* normal at the previous step (history) */
    double fn;             /* normal force magnitude (last step) */
    double n[3], cp[3], pen;
} orc_contact;

struct orc_scene {
    long n, cap;
    double *pos, *vel, *angvel, *ori, *radius, *mass, *inertia, *force, *torque;
    int *mat;
    unsigned char *fixed;
    orc_mat mats[ORC_MAX_MAT];
    int periodic;
    double H[9], Hprev[9], L[9], Lprev[9], Lnext[9];
    int L_pending;
    double box_lo[3], box_hi[3];
    int wall_mask;
    double g[3], damping, dt;
    long iter;
    double time;
    orc_contact *con;
    long ncon, capcon;
    /* energy tracker (cumulative works) */
    double grav_work, nonvisc_damp, plast_dissip;
    /* stress-controlled periodic cell (PeriTriaxController reading R16) */
    int triax, stress_mask, glob_update;
    /* contact law: 0 Law2_ScGeom_FrictPhys_CundallStrack, 1 Hertz-Mindlin (R18) */
    int law;
    /* GlobalStiffnessTimeStepper (R17) */
    int tstep, tstep_interval;
    double tstep_safety, tstep_default, tstep_max;
    /* density scaling (reading R22): per-body inertia factor f, target step */
    int dscale_on;
    double target_dt;
    double *dscale;
    double goal[3], max_rate[3], grow_damping;
    /* Peri3dController (reading R23) */
    int p3d, p3d_mask, p3d_first, p3d_done;
    long p3d_nsteps, p3d_k;
    double p3d_goal[6], p3d_mod, p3d_max_rate, p3d_young, p3d_poisson, p3d_max_strain;
    int p3d_npath[6];
    double p3d_path[6][16][2];
    double p3d_rate[6], p3d_err[6], p3d_H0[9], p3d_T0[9], p3d_stress[6], p3d_strain[6];
};

/* ---------------------------------------------------------------- vectors */
static void v_cross(const double *a, const double *b, double *o) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double v_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void m_vec(const double *M, const double *v, double *o) { /* o = M v, row-major */
    double x = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    double y = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
    double z = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
    o[0] = x; o[1] = y; o[2] = z;
}
static void m_mul(const double *A, const double *B, double *O) {
    double T[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            T[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
    memcpy(O, T, sizeof T);
}
static double m_det(const double *M) {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}
static int m_inv(const double *M, double *O) { /* Cramer's rule */
    double d = m_det(M);
    if (d == 0 || !isfinite(d)) return -1;
    double T[9];
    T[0] = (M[4] * M[8] - M[5] * M[7]) / d;
    T[1] = (M[2] * M[7] - M[1] * M[8]) / d;
    T[2] = (M[1] * M[5] - M[2] * M[4]) / d;
    T[3] = (M[5] * M[6] - M[3] * M[8]) / d;
    T[4] = (M[0] * M[8] - M[2] * M[6]) / d;
    T[5] = (M[2] * M[3] - M[0] * M[5]) / d;
    T[6] = (M[3] * M[7] - M[4] * M[6]) / d;
    T[7] = (M[1] * M[6] - M[0] * M[7]) / d;
    T[8] = (M[0] * M[4] - M[1] * M[3]) / d;
    memcpy(O, T, sizeof T);
    return 0;
}
static double sgn(double x) { return (x > 0) - (x < 0); }

/* Image shift h = H c of the periodic cell (section 2.1.6: cellDist times cell). */
static void cell_shift(const double *H, const int *c, double *h) {
    double cd[3] = {(double)c[0], (double)c[1], (double)c[2]};
    m_vec(H, cd, h);
}

/* Branch vector d = (x2 + H c) - x1 and its squared length.  This is the exact
 * test of the two-pass detection (eq. 2.2 second pass): real iff d2 < (r1+r2)^2. */
static double branch(const double *x1, const double *x2, const double *h, double *d) {
    for (int k = 0; k < 3; ++k) d[k] = (x2[k] + h[k]) - x1[k];
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

/* Minimum-image shift c for the pair (x1, x2): c = -round(H^-1 (x2 - x1)). */
static void min_image(const double *Hinv, const double *x1, const double *x2, int *c) {
    double d[3] = {x2[0] - x1[0], x2[1] - x1[1], x2[2] - x1[2]}, s[3];
    m_vec(Hinv, d, s);
    for (int k = 0; k < 3; ++k) c[k] = -(int)floor(s[k] + 0.5);
}

/* Perpendicular widths of the cell (distance between opposite faces). */
static void cell_widths(const double *H, double *w) {
    double a[3] = {H[0], H[3], H[6]}, b[3] = {H[1], H[4], H[7]}, cc[3] = {H[2], H[5], H[8]};
    double V = fabs(m_det(H)), x[3];
    v_cross(b, cc, x); w[0] = V / sqrt(v_dot(x, x));
    v_cross(cc, a, x); w[1] = V / sqrt(v_dot(x, x));
    v_cross(a, b, x); w[2] = V / sqrt(v_dot(x, x));
}

/* ------------------------------------------------------------ pair search */
typedef struct { int i, j, c[3]; } orc_pair;

static int pair_cmp(const void *a, const void *b) {
    const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
    if (x->i != y->i) return (x->i < y->i) ? -1 : 1;
    if (x->j != y->j) return (x->j < y->j) ? -1 : 1;
    for (int k = 0; k < 3; ++k)
        if (x->c[k] != y->c[k]) return (x->c[k] < y->c[k]) ? -1 : 1;
    return 0;
}

typedef struct { orc_pair *p; long n, cap; int oom; } pair_list;

static void pl_push(pair_list *L, int i, int j, const int *c) {
    if (L->n == L->cap) {
        long nc = L->cap ? 2 * L->cap : 1024;
        orc_pair *q = (orc_pair *)realloc(L->p, nc * sizeof(orc_pair));
        if (!q) { L->oom = 1; return; }
        L->p = q; L->cap = nc;
    }
    orc_pair *e = &L->p[L->n++];
    e->i = i; e->j = j; e->c[0] = c[0]; e->c[1] = c[1]; e->c[2] = c[2];
}

/* Test one unordered pair (a, b): orient as (min id, max id), take the minimum
 * image in a periodic cell, keep it when |d| < r_a + r_b + margin. */
static void test_pair(long a, long b, const double *pos, const double *rad, int periodic,
                      const double *H, const double *Hinv, double margin, pair_list *out) {
    long i = a < b ? a : b, j = a < b ? b : a;
    int c[3] = {0, 0, 0};
    double h[3] = {0, 0, 0}, d[3];
    if (periodic) { min_image(Hinv, pos + 3 * i, pos + 3 * j, c); cell_shift(H, c, h); }
    double d2 = branch(pos + 3 * i, pos + 3 * j, h, d);
    double R = (rad[i] + rad[j]) + margin;
    if (d2 < R * R) pl_push(out, (int)i, (int)j, c);
}

static long pairs_out(pair_list *L, long cap, int *I, int *J, int *C) {
    if (L->oom) { free(L->p); return -2; }
    qsort(L->p, L->n, sizeof(orc_pair), pair_cmp);
    /* a periodic sweep window may see one pair from both ends: drop repeats */
    long m = 0;
    for (long k = 0; k < L->n; ++k)
        if (m == 0 || pair_cmp(&L->p[m - 1], &L->p[k]) != 0) L->p[m++] = L->p[k];
    for (long k = 0; k < m && k < cap; ++k) {
        I[k] = L->p[k].i; J[k] = L->p[k].j;
        if (C) { C[3 * k] = L->p[k].c[0]; C[3 * k + 1] = L->p[k].c[1]; C[3 * k + 2] = L->p[k].c[2]; }
    }
    free(L->p);
    return m;
}

long orc_pairs_bruteforce(long n, const double *pos, const double *radius, int periodic,
                          const double *H9, double margin, long cap, int *I, int *J, int *C) {
    double Hinv[9];
    if (periodic && m_inv(H9, Hinv) != 0) return -1;
    pair_list L = {0};
    for (long a = 0; a < n; ++a)
        for (long b = a + 1; b < n; ++b)
            test_pair(a, b, pos, radius, periodic, H9, Hinv, margin, &L);
    return pairs_out(&L, cap, I, J, C);
}

typedef struct { double key; long id; } sweep_item;
static int sweep_cmp(const void *a, const void *b) {
    const sweep_item *x = (const sweep_item *)a, *y = (const sweep_item *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Sort-and-sweep along the first axis (section 2.1.1, "Sweep and prune": sort
 * the bounds, traverse each body's range, test the overlaps found).  Periodic
 * cells sweep the wrapped fractional coordinate with a circular window. */
static long sweep_core(long n, const double *pos, const double *radius, int periodic,
                       const double *H9, double margin, pair_list *L) {
    if (n <= 0) return 0;
    double Hinv[9];
    if (periodic && m_inv(H9, Hinv) != 0) return -1;
    double rmax = 0;
    for (long i = 0; i < n; ++i) if (radius[i] > rmax) rmax = radius[i];
    sweep_item *it = (sweep_item *)malloc(sizeof(sweep_item) * n);
    if (!it) return -2;
    if (!periodic) {
        /* lower bound of each (enlarged) Aabb along x; a tiny relative pad keeps the
         * filter conservative against rounding, the exact test decides */
        for (long i = 0; i < n; ++i) {
            double e = radius[i] + 0.5 * margin;
            it[i].key = pos[3 * i] - e - 1e-9 * e;
            it[i].id = i;
        }
        qsort(it, n, sizeof(sweep_item), sweep_cmp);
        for (long a = 0; a < n; ++a) {
            long i = it[a].id;
            double e = radius[i] + 0.5 * margin;
            double hi = pos[3 * i] + e + 1e-9 * e;
            for (long b = a + 1; b < n && it[b].key < hi; ++b)
                test_pair(i, it[b].id, pos, radius, 0, H9, Hinv, margin, L);
        }
    } else {
        /* fractional coordinate s0 = (H^-1 x)_0 wrapped into [0,1); a displacement
         * of length r moves s0 by at most r*|row0(H^-1)| */
        double g = sqrt(Hinv[0] * Hinv[0] + Hinv[1] * Hinv[1] + Hinv[2] * Hinv[2]);
        for (long i = 0; i < n; ++i) {
            const double *x = pos + 3 * i;
            double s = Hinv[0] * x[0] + Hinv[1] * x[1] + Hinv[2] * x[2];
            it[i].key = s - floor(s);
            it[i].id = i;
        }
        qsort(it, n, sizeof(sweep_item), sweep_cmp);
        for (long a = 0; a < n; ++a) {
            long i = it[a].id;
            double w = (radius[i] + rmax + margin) * g * (1 + 1e-9) + 1e-15;
            if (w >= 0.5) w = 0.5; /* the whole circle is within reach */
            for (long k = 1; k < n; ++k) {
                long b = (a + k) % n;
                double ds = it[b].key - it[a].key;
                if (ds < 0) ds += 1.0;
                if (ds > w) break;
                test_pair(i, it[b].id, pos, radius, 1, H9, Hinv, margin, L);
            }
        }
    }
    free(it);
    return 0;
}

long orc_pairs_sweep(long n, const double *pos, const double *radius, int periodic,
                     const double *H9, double margin, long cap, int *I, int *J, int *C) {
    pair_list L = {0};
    long rc = sweep_core(n, pos, radius, periodic, H9, margin, &L);
    if (rc < 0) { free(L.p); return rc; }
    return pairs_out(&L, cap, I, J, C);
}

/* Cell-list search: bodies hashed into a uniform grid whose cells are at least as
 * wide as the largest possible contact distance (2 r_max + margin), each body
 * tested against the bodies of its own and the 26 neighbouring cells.  In a
 * periodic cell the grid lives in wrapped fractional coordinates, sized by the
 * perpendicular widths.  Every candidate goes through test_pair, so the result is
 * the same set as the brute-force search. */
static long grid_core(long n, const double *pos, const double *radius, int periodic,
                      const double *H9, double margin, pair_list *L) {
    if (n <= 0) return 0;
    double Hinv[9];
    if (periodic && m_inv(H9, Hinv) != 0) return -1;
    double rmax = 0;
    for (long i = 0; i < n; ++i) if (radius[i] > rmax) rmax = radius[i];
    double reach = (2 * rmax + margin) * (1 + 1e-9) + 1e-300;
    double lo[3] = {0, 0, 0}, ext[3];
    int nc[3];
    if (periodic) {
        double w[3];
        cell_widths(H9, w);
        for (int k = 0; k < 3; ++k) {
            nc[k] = (int)floor(w[k] / reach);
            if (nc[k] < 1) nc[k] = 1;
            if (nc[k] > 512) nc[k] = 512;
            ext[k] = 1.0;
        }
    } else {
        double hi[3];
        for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
        for (long i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                if (pos[3 * i + k] < lo[k]) lo[k] = pos[3 * i + k];
                if (pos[3 * i + k] > hi[k]) hi[k] = pos[3 * i + k];
            }
        for (int k = 0; k < 3; ++k) {
            ext[k] = hi[k] - lo[k];
            nc[k] = (int)floor(ext[k] / reach);
            if (nc[k] < 1) nc[k] = 1;
            if (nc[k] > 512) nc[k] = 512;
            if (ext[k] <= 0) ext[k] = 1;
        }
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    long *head = (long *)malloc(sizeof(long) * ncell);
    long *next = (long *)malloc(sizeof(long) * n);
    int *cell = (int *)malloc(sizeof(int) * 3 * n);
    if (!head || !next || !cell) { free(head); free(next); free(cell); return -2; }
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (long i = n - 1; i >= 0; --i) {
        double u[3];
        if (periodic) {
            m_vec(Hinv, pos + 3 * i, u);
            for (int k = 0; k < 3; ++k) u[k] = u[k] - floor(u[k]);
        } else {
            for (int k = 0; k < 3; ++k) u[k] = (pos[3 * i + k] - lo[k]) / ext[k];
        }
        for (int k = 0; k < 3; ++k) {
            int c = (int)floor(u[k] * nc[k]);
            if (c < 0) c = 0;
            if (c >= nc[k]) c = nc[k] - 1;
            cell[3 * i + k] = c;
        }
        long id = ((long)cell[3 * i] * nc[1] + cell[3 * i + 1]) * nc[2] + cell[3 * i + 2];
        next[i] = head[id];
        head[id] = i;
    }
    for (long i = 0; i < n; ++i) {
        int nb[3][3], nnb[3];
        for (int k = 0; k < 3; ++k) {
            nnb[k] = 0;
            for (int d = -1; d <= 1; ++d) {
                int c = cell[3 * i + k] + d;
                if (periodic) { c %= nc[k]; if (c < 0) c += nc[k]; }
                else if (c < 0 || c >= nc[k]) continue;
                int dup = 0;
                for (int q = 0; q < nnb[k]; ++q) if (nb[k][q] == c) dup = 1;
                if (!dup) nb[k][nnb[k]++] = c;
            }
        }
        for (int a = 0; a < nnb[0]; ++a)
            for (int b = 0; b < nnb[1]; ++b)
                for (int c = 0; c < nnb[2]; ++c) {
                    long id = ((long)nb[0][a] * nc[1] + nb[1][b]) * nc[2] + nb[2][c];
                    for (long j = head[id]; j >= 0; j = next[j])
                        if (j > i) test_pair(i, j, pos, radius, periodic, H9, Hinv, margin, L);
                }
    }
    free(head); free(next); free(cell);
    return L->oom ? -2 : 0;
}

long orc_pairs_grid(long n, const double *pos, const double *radius, int periodic,
                    const double *H9, double margin, long cap, int *I, int *J, int *C) {
    pair_list L = {0};
    long rc = grid_core(n, pos, radius, periodic, H9, margin, &L);
    if (rc < 0) { free(L.p); return rc; }
    return pairs_out(&L, cap, I, J, C);
}

/* --------------------------------------------------------------- scene */
orc_scene *orc_create(int periodic, const double *H9, const double *box_lo, const double *box_hi,
                      int wall_mask, const double *gravity, double damping, double dt) {
    orc_scene *s = (orc_scene *)calloc(1, sizeof(orc_scene));
    if (!s) return NULL;
    s->periodic = periodic ? 1 : 0;
    for (int k = 0; k < 9; ++k) s->H[k] = H9 ? H9[k] : (k % 4 == 0);
    memcpy(s->Hprev, s->H, sizeof s->H);
    for (int k = 0; k < 3; ++k) {
        s->box_lo[k] = box_lo ? box_lo[k] : 0;
        s->box_hi[k] = box_hi ? box_hi[k] : 1;
        s->g[k] = gravity ? gravity[k] : 0;
    }
    s->wall_mask = periodic ? 0 : (wall_mask & 0x3F);
    s->damping = damping;
    s->dt = dt;
    if (s->periodic && fabs(m_det(s->H)) == 0) { free(s); return NULL; }
    return s;
}

static void free_bodies(orc_scene *s) {
    free(s->pos); free(s->vel); free(s->angvel); free(s->ori); free(s->radius); free(s->mass);
    free(s->inertia); free(s->force); free(s->torque); free(s->mat); free(s->fixed);
    free(s->dscale);
}

void orc_destroy(orc_scene *s) {
    if (!s) return;
    free_bodies(s);
    free(s->con);
    free(s);
}

int orc_set_material(orc_scene *s, int mat, double density, double young, double poisson,
                     double friction_angle) {
    if (!s || mat < 0 || mat >= ORC_MAX_MAT) return -1;
    if (!(density > 0) || !(young > 0) || !(poisson >= 0) || !(friction_angle >= 0) ||
        !(friction_angle < 1.5707963267948966))
        return -1;
    orc_mat *m = &s->mats[mat];
    m->density = density; m->young = young; m->poisson = poisson; m->friction = friction_angle;
    m->set = 1;
    return 0;
}

static int grow(orc_scene *s, long need) {
    if (need <= s->cap) return 0;
    long nc = s->cap ? s->cap : 64;
    while (nc < need) nc *= 2;
#define GROW(p, T, k)                                                                     \
    do {                                                                                  \
        T *q = (T *)realloc(s->p, sizeof(T) * (k) * nc);                                 \
        if (!q) return -2;                                                                \
        s->p = q;                                                                         \
    } while (0)
    GROW(pos, double, 3); GROW(vel, double, 3); GROW(angvel, double, 3); GROW(ori, double, 4);
    GROW(radius, double, 1); GROW(mass, double, 1); GROW(inertia, double, 1);
    GROW(force, double, 3); GROW(torque, double, 3); GROW(mat, int, 1);
    GROW(fixed, unsigned char, 1); GROW(dscale, double, 1);
#undef GROW
    s->cap = nc;
    return 0;
}

long orc_add_spheres(orc_scene *s, long n, const double *pos, const double *radius,
                     const int *mat, const double *vel, const double *angvel,
                     const unsigned char *fixed) {
    if (!s || n < 0 || (n > 0 && (!pos || !radius))) return -1;
    for (long i = 0; i < n; ++i) {
        int m = mat ? mat[i] : 0;
        if (m < 0 || m >= ORC_MAX_MAT || !s->mats[m].set) return -1;
        if (!(radius[i] > 0) || !isfinite(radius[i])) return -1;
        for (int k = 0; k < 3; ++k) if (!isfinite(pos[3 * i + k])) return -1;
    }
    if (grow(s, s->n + n)) return -2;
    const double pi = 3.14159265358979323846;
    for (long t = 0; t < n; ++t) {
        long i = s->n + t;
        int m = mat ? mat[t] : 0;
        double r = radius[t];
        for (int k = 0; k < 3; ++k) {
            s->pos[3 * i + k] = pos[3 * t + k];
            s->vel[3 * i + k] = vel ? vel[3 * t + k] : 0;
            s->angvel[3 * i + k] = angvel ? angvel[3 * t + k] : 0;
            s->force[3 * i + k] = 0;
            s->torque[3 * i + k] = 0;
        }
        s->ori[4 * i] = 1; s->ori[4 * i + 1] = 0; s->ori[4 * i + 2] = 0; s->ori[4 * i + 3] = 0;
        s->radius[i] = r;
        s->mat[i] = m;
        s->fixed[i] = fixed ? (fixed[t] != 0) : 0;
        /* utils.sphere: mass from density and volume, inertia of a solid sphere (R12) */
        s->mass[i] = s->mats[m].density * (4.0 / 3.0) * pi * r * r * r;
        s->inertia[i] = 0.4 * s->mass[i] * r * r;
        s->dscale[i] = 1.0;
    }
    long first = s->n;
    s->n += n;
    return first;
}

int orc_set_dt(orc_scene *s, double dt) {
    if (!s || !(dt > 0)) return -1;
    s->dt = dt;
    return 0;
}

/* Cell.velGrad: the assignment is deferred and takes effect at the next step
 * (Cell class reference, "velGrad" note; nextVelGrad). */
int orc_set_velgrad(orc_scene *s, const double *L9) {
    if (!s || !s->periodic) return -1;
    memcpy(s->Lnext, L9, sizeof s->Lnext);
    s->L_pending = 1;
    return 0;
}

/* utils.SpherePWaveTimeStep: dt = r / sqrt(E / rho) (section 2.1.5 "Stability
 * considerations", estimate by p-wave propagation speed). */
double orc_sphere_pwave_dt(double radius, double density, double young) {
    return radius / sqrt(young / density);
}

/* utils.PWaveTimeStep: the minimum over all spheres. */
double orc_pwave_dt(const orc_scene *s) {
    double dt = INFINITY;
    for (long i = 0; i < s->n; ++i) {
        const orc_mat *m = &s->mats[s->mat[i]];
        double d = orc_sphere_pwave_dt(s->radius[i], m->density, m->young);
        if (d < dt) dt = d;
    }
    return dt;
}

/* Ip2_FrictMat_FrictMat_FrictPhys: contact stiffness of two springs in series,
 * k = k1 k2 / (k1 + k2) with k_i = E_i * (2 r_i); shear stiffness with E_i * nu_i;
 * friction angle min(phi1, phi2) (section 2.1.2 and class reference). */
static void ip2_frict(const orc_mat *m1, double r1, const orc_mat *m2, double r2, double *kn,
                      double *ks, double *tanphi) {
    double k1 = m1->young * (2 * r1), k2 = m2->young * (2 * r2);
    *kn = k1 * k2 / (k1 + k2);
    double s1 = m1->young * m1->poisson * (2 * r1), s2 = m2->young * m2->poisson * (2 * r2);
    *ks = s1 * s2 / (s1 + s2);
    double phi = m1->friction < m2->friction ? m1->friction : m2->friction;
    *tanphi = tan(phi);
}

/* Ip2_FrictMat_FrictMat_MindlinPhys (class reference; reading R18): Hertz normal
 * constant kno = 4/3 E* sqrt(R*) and Mindlin shear constant kso, with the textbook
 * combinations 1/E* = (1 - nu1^2)/E1 + (1 - nu2^2)/E2, R* = r1 r2 / (r1 + r2) (a wall
 * is an infinite radius: r2 < 0 gives R* = r1), G_i = E_i / (2 (1 + nu_i)) and
 * kso = 8 sqrt(R*) / ((2 - nu1)/G1 + (2 - nu2)/G2), which is the text's
 * 2 sqrt(4R) G / (2 - nu) for equal materials.  The FrictMat "poisson" is the true
 * Poisson ratio here (ElastMat reference). */
static void ip2_mindlin(const orc_mat *m1, double r1, const orc_mat *m2, double r2,
                        double *kno, double *kso, double *tanphi) {
    double Es = 1.0 / ((1 - m1->poisson * m1->poisson) / m1->young +
                       (1 - m2->poisson * m2->poisson) / m2->young);
    double Rs = r2 < 0 ? r1 : r1 * r2 / (r1 + r2);
    double G1 = m1->young / (2 * (1 + m1->poisson)), G2 = m2->young / (2 * (1 + m2->poisson));
    *kno = 4.0 / 3.0 * Es * sqrt(Rs);
    *kso = 8.0 * sqrt(Rs) / ((2 - m1->poisson) / G1 + (2 - m2->poisson) / G2);
    double phi = m1->friction < m2->friction ? m1->friction : m2->friction;
    *tanphi = tan(phi);
}

/* tangent stiffnesses of a contact at penetration pen (the Hertz-Mindlin constants
 * are stored in kn, ks: k_n = 3/2 kno pen^1/2, k_s = kso pen^1/2) */
static void tangent_stiffness(const orc_scene *s, const orc_contact *ct, double *kn, double *ks) {
    if (s->law == 1) {
        double sq = sqrt(ct->pen > 0 ? ct->pen : 0.0);
        *kn = 1.5 * ct->kn * sq;
        *ks = ct->ks * sq;
    } else {
        *kn = ct->kn;
        *ks = ct->ks;
    }
}

int orc_set_law(orc_scene *s, int law) {
    if (!s || (law != 0 && law != 1)) return -1;
    s->law = law;
    return 0;
}

/* One contact: given the current normal n, penetration pen, contact point, the
 * velocities at the contact and the FrictPhys, update the shear force and
 * return the force on body 2 (sections 2.1.3 and 2.1.4). */
static void shear_and_law(orc_contact *ct, const double *n, double pen, const double *v1,
                          const double *w1, const double *v2, const double *w2, double r1,
                          double r2, double l, double dt, int law, double *F2, double *plast) {
    /* Hertz-Mindlin (R18): Fn = kno pen^3/2 and the shear spring at ks = kso pen^1/2 */
    double sq = law == 1 ? sqrt(pen) : 1.0;
    double ks = law == 1 ? ct->ks * sq : ct->ks;
    /* 1. motion of the contact frame: both increments from the previous value (R5) */
    double a[3], tn[3], d1[3], d2[3], fs[3];
    v_cross(ct->nprev, n, a);                               /* n- x n */
    double ws[3] = {w1[0] + w2[0], w1[1] + w2[1], w1[2] + w2[2]};
    double tw = 0.5 * dt * v_dot(n, ws);                    /* dt/2 n.(w1+w2) */
    for (int k = 0; k < 3; ++k) tn[k] = tw * n[k];
    v_cross(ct->fs, a, d1);
    v_cross(ct->fs, tn, d2);
    for (int k = 0; k < 3; ++k) fs[k] = ct->fs[k] - d1[k] - d2[k];
    /* 2. mutual motion (ScGeom relative velocity, R3), its part perpendicular to n */
    double rr[3], cr[3], v12[3];
    for (int k = 0; k < 3; ++k) rr[k] = r2 * w2[k] + r1 * w1[k];
    v_cross(rr, n, cr);
    double f = (r1 + r2) / l;
    for (int k = 0; k < 3; ++k) v12[k] = f * (v2[k] - v1[k]) - cr[k];
    double vn = v_dot(n, v12);
    double v12s[3];
    for (int k = 0; k < 3; ++k) v12s[k] = v12[k] - vn * n[k];
    /* shear spring increment on body 2 (R2) */
    for (int k = 0; k < 3; ++k) fs[k] = fs[k] - ks * (dt * v12s[k]);
    /* Law2_ScGeom_FrictPhys_CundallStrack: Fn = kn pen, Coulomb cap */
    double Fn = law == 1 ? ct->kn * pen * sq : ct->kn * pen;
    double maxFs = Fn * ct->tanphi;
    double fs2 = v_dot(fs, fs);
    if (fs2 > maxFs * maxFs) {
        double trial[3] = {fs[0], fs[1], fs[2]};
        double scale = maxFs / sqrt(fs2);
        for (int k = 0; k < 3; ++k) fs[k] = fs[k] * scale;
        /* slip work (trial - final)/ks . final */
        double dd[3] = {trial[0] - fs[0], trial[1] - fs[1], trial[2] - fs[2]};
        *plast += v_dot(dd, fs) / ks;
    }
    for (int k = 0; k < 3; ++k) {
        ct->fs[k] = fs[k];
        ct->nprev[k] = n[k];
        ct->n[k] = n[k];
        F2[k] = Fn * n[k] + fs[k];
    }
    ct->fn = Fn;
    ct->pen = pen;
}

/* walls: index w = 2*axis + side; side 0 at box_lo, side 1 at box_hi */
static double wall_coord(const orc_scene *s, int w) {
    return (w & 1) ? s->box_hi[w >> 1] : s->box_lo[w >> 1];
}

typedef struct { int id1, id2, c[3]; } orc_key;

static int key_cmp_contact(const orc_key *k, const orc_contact *c) {
    if (k->id1 != c->id1) return (k->id1 < c->id1) ? -1 : 1;
    if (k->id2 != c->id2) return (k->id2 < c->id2) ? -1 : 1;
    return 0;
}

/* Collider + potential/real bookkeeping: the set of real interactions of this
 * step, each carrying its history from the previous step when the same pair
 * (same cell shift) was already real, else marked new (kn = 0). */
static int detect_contacts(orc_scene *s, orc_contact **out, long *nout) {
    pair_list L = {0};
    long rc = grid_core(s->n, s->pos, s->radius, s->periodic, s->H, 0.0, &L);
    if (rc < 0 || L.oom) { free(L.p); return rc < 0 ? (int)rc : -2; }
    qsort(L.p, L.n, sizeof(orc_pair), pair_cmp);
    long m = 0;
    for (long k = 0; k < L.n; ++k)
        if (m == 0 || pair_cmp(&L.p[m - 1], &L.p[k]) != 0) L.p[m++] = L.p[k];
    /* wall contacts: pen = r - |x_a - w| > 0 (R10) */
    long nw = 0;
    orc_key *wk = NULL;
    if (s->wall_mask) {
        wk = (orc_key *)malloc(sizeof(orc_key) * (6 * s->n + 1));
        if (!wk) { free(L.p); return -2; }
        for (int w = 0; w < 6; ++w) {
            if (!(s->wall_mask & (1 << w))) continue;
            double wc = wall_coord(s, w);
            for (long i = 0; i < s->n; ++i) {
                double dist = s->pos[3 * i + (w >> 1)] - wc;
                if (fabs(dist) < s->radius[i]) {
                    orc_key *e = &wk[nw++];
                    e->id1 = -(w + 1); e->id2 = (int)i; e->c[0] = e->c[1] = e->c[2] = 0;
                }
            }
        }
    }
    long total = nw + m;
    orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (total + 1));
    orc_contact *nc = (orc_contact *)calloc(total + 1, sizeof(orc_contact));
    if (!keys || !nc) { free(L.p); free(wk); free(keys); free(nc); return -2; }
    /* canonical order: walls (negative id1, most negative first) then sphere pairs */
    long t = 0;
    for (int w = 5; w >= 0; --w)
        for (long k = 0; k < nw; ++k) if (wk[k].id1 == -(w + 1)) keys[t++] = wk[k];
    for (long k = 0; k < m; ++k) {
        keys[t].id1 = L.p[k].i; keys[t].id2 = L.p[k].j;
        for (int q = 0; q < 3; ++q) keys[t].c[q] = L.p[k].c[q];
        ++t;
    }
    free(L.p);
    free(wk);
    /* merge with the previous list (both sorted by (id1, id2)) */
    long o = 0;
    for (long k = 0; k < total; ++k) {
        orc_contact *c = &nc[k];
        while (o < s->ncon && key_cmp_contact(&keys[k], &s->con[o]) > 0) ++o;
        if (o < s->ncon && key_cmp_contact(&keys[k], &s->con[o]) == 0 &&
            s->con[o].c[0] == keys[k].c[0] && s->con[o].c[1] == keys[k].c[1] &&
            s->con[o].c[2] == keys[k].c[2]) {
            *c = s->con[o];
        } else {
            memset(c, 0, sizeof *c);
            c->id1 = keys[k].id1; c->id2 = keys[k].id2;
            for (int q = 0; q < 3; ++q) c->c[q] = keys[k].c[q];
            c->kn = 0; /* new: Ip2 runs below */
        }
    }
    free(keys);
    *out = nc;
    *nout = total;
    return 0;
}

static int check_cell(const orc_scene *s) {
    if (!s->periodic) return 0;
    double w[3], rmax = 0;
    cell_widths(s->H, w);
    for (long i = 0; i < s->n; ++i) if (s->radius[i] > rmax) rmax = s->radius[i];
    /* a sphere pair must not span more than half the cell (section 2.1.6) */
    for (int k = 0; k < 3; ++k) if (!(2 * rmax < 0.5 * w[k])) return -3;
    return 0;
}

static void quat_mul(const double *a, const double *b, double *o) { /* (w,x,y,z) */
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

/* PeriTriaxController servo, reading R16. */
static void triax_update(orc_scene *s) {
    double V = fabs(m_det(s->Hprev));   /* the cell the contacts of this step were computed in */
    double sig[3] = {0, 0, 0}, K[3] = {0, 0, 0};
    for (long k = 0; k < s->ncon; ++k) {
        const orc_contact *ct = &s->con[k];
        if (ct->id1 < 0) continue;
        double l = (s->radius[ct->id1] + s->radius[ct->id2]) - ct->pen;
        for (int a = 0; a < 3; ++a) {
            double F = ct->fn * ct->n[a] + ct->fs[a];
            sig[a] += F * (-l * ct->n[a]);
            double b = l * ct->n[a];
            double kt, kst;
            tangent_stiffness(s, ct, &kt, &kst);
            K[a] += kt * (b * b);
        }
    }
    double L[9];
    memcpy(L, s->L_pending ? s->Lnext : s->L, sizeof L);
    for (int a = 0; a < 3; ++a) {
        double rate;
        if (s->stress_mask & (1 << a)) {
            double sa = sig[a] / V, Ka = K[a] / V;
            double want = (1 - s->grow_damping) * (s->goal[a] - sa);
            if (Ka > 0) rate = want / (Ka * (s->dt * s->glob_update));
            else rate = want > 0 ? s->max_rate[a] : (want < 0 ? -s->max_rate[a] : 0.0);
            if (rate > s->max_rate[a]) rate = s->max_rate[a];
            if (rate < -s->max_rate[a]) rate = -s->max_rate[a];
        } else {
            rate = s->goal[a];
        }
        L[4 * a] = rate;
    }
    memcpy(s->Lnext, L, sizeof L);
    s->L_pending = 1;
}

/* ------------------------------------------------------------ Peri3dController */
/* Voigt order of the six components: xx, yy, zz, yz, zx, xy (the attribute order of
 * goal, stress and strain; stressMask bit i = component i). */
static const int VO[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {2, 0}, {0, 1}};

/* Prescribed value of component i at progress p (xxPath ... "time functions"):
 * couples (t_j, v_j), the last one standing for (nSteps, goal), the others scaled
 * by it; piecewise linear from (0, 0); the goal beyond the last couple. */
static double p3d_path_value(const orc_scene *s, int i, double p) {
    const int n = s->p3d_npath[i];
    const double tl = s->p3d_path[i][n - 1][0], vl = s->p3d_path[i][n - 1][1];
    double t0 = 0, v0 = 0;
    for (int j = 0; j < n; ++j) {
        const double t1 = s->p3d_path[i][j][0] / tl, v1 = s->p3d_path[i][j][1] / vl;
        if (p <= t1) {
            const double a = t1 > t0 ? (p - t0) / (t1 - t0) : 1.0;
            return s->p3d_goal[i] * (v0 + a * (v1 - v0));
        }
        t0 = t1; v0 = v1;
    }
    return s->p3d_goal[i];
}

/* Polar decomposition T = U P (U a rotation, P symmetric) by the iteration
 * X <- (X + X^-T) / 2 from X = T, which converges to U for det T > 0. */
static void polar(const double *T, double *U, double *P) {
    double X[9], Xi[9];
    memcpy(X, T, sizeof X);
    for (int it = 0; it < 60; ++it) {
        if (m_inv(X, Xi)) break;
        double Y[9], d = 0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Y[3 * r + c] = 0.5 * (X[3 * r + c] + Xi[3 * c + r]);
        for (int q = 0; q < 9; ++q) d += fabs(Y[q] - X[q]);
        memcpy(X, Y, sizeof X);
        if (d < 1e-15) break;
    }
    memcpy(U, X, sizeof X);
    double Ut[9], Pm[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ut[3 * r + c] = U[3 * c + r];
    m_mul(Ut, T, Pm);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) P[3 * r + c] = 0.5 * (Pm[3 * r + c] + Pm[3 * c + r]);
}

/* One controller update at the end of a step (reading R23): stress and strain now,
 * the next strain rates, and the velocity gradient that realises them over the next
 * step (assigned like Cell.velGrad). */
static void p3d_update(orc_scene *s) {
    const double dt = s->dt;
    /* stress of this step's contacts (Love-Weber, compression negative), symmetrised */
    double V = fabs(m_det(s->Hprev)), S[9] = {0};
    for (long k = 0; k < s->ncon; ++k) {
        const orc_contact *ct = &s->con[k];
        if (ct->id1 < 0) continue;
        double l = (s->radius[ct->id1] + s->radius[ct->id2]) - ct->pen;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                S[3 * a + b] += (ct->fn * ct->n[a] + ct->fs[a]) * (-l * ct->n[b]);
    }
    /* Cell.trsf: T = H H0^-1 T0 (T0 the transformation at the start) = U P; the strain
     * P - I rotated back to global axes, U (P - I) U^T */
    double H0i[9], T1[9], T[9], U[9], P[9], Pm[9], Ut[9], G1[9], G[9];
    m_inv(s->p3d_H0, H0i);
    m_mul(s->H, H0i, T1);
    m_mul(T1, s->p3d_T0, T);
    polar(T, U, P);
    for (int q = 0; q < 9; ++q) Pm[q] = P[q] - (q % 4 == 0 ? 1.0 : 0.0);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ut[3 * r + c] = U[3 * c + r];
    m_mul(U, Pm, G1);
    m_mul(G1, Ut, G);
    double sig[6], eps[6];
    for (int i = 0; i < 6; ++i) {
        const int a = VO[i][0], b = VO[i][1];
        sig[i] = 0.5 * (S[3 * a + b] + S[3 * b + a]) / V;
        eps[i] = a == b ? G[3 * a + a] : G[3 * a + b] + G[3 * b + a];   /* engineering shear */
        s->p3d_stress[i] = sig[i];
        s->p3d_strain[i] = eps[i];
    }
    if (s->p3d_done) return;
    const long k = ++s->p3d_k;
    double emax = 0;
    for (int i = 0; i < 6; ++i) if (fabs(eps[i]) > emax) emax = fabs(eps[i]);
    if (k >= s->p3d_nsteps || emax >= s->p3d_max_strain) { s->p3d_done = 1; return; }
    const double p = (double)k / s->p3d_nsteps, pn = (double)(k + 1) / s->p3d_nsteps;
    double rate[6], err[6], rmax = 0;
    for (int i = 0; i < 6; ++i) if (fabs(s->p3d_rate[i]) > rmax) rmax = fabs(s->p3d_rate[i]);
    for (int i = 0; i < 6; ++i) {
        rate[i] = s->p3d_rate[i];
        err[i] = 0;
        if (!(s->p3d_mask & (1 << i))) {          /* strain: the rate that reaches the path */
            rate[i] = (p3d_path_value(s, i, pn) - eps[i]) / dt;
        } else {
            err[i] = sig[i] - p3d_path_value(s, i, p);
        }
    }
    if (s->p3d_first) {
        /* first update: stress components from an isotropic elastic estimate, the
         * strain components as prescribed: D_SS de_S = dsig_S - D_SE de_E */
        const double E = s->p3d_young, nu = s->p3d_poisson;
        const double lam = E * nu / ((1 + nu) * (1 - 2 * nu)), G = E / (2 * (1 + nu));
        double D[6][6] = {{0}};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) D[i][j] = lam;
            D[i][i] = lam + 2 * G;
            D[3 + i][3 + i] = G;
        }
        int idx[6], m = 0;
        for (int i = 0; i < 6; ++i) if (s->p3d_mask & (1 << i)) idx[m++] = i;
        double A[6][7];
        for (int r = 0; r < m; ++r) {
            const int i = idx[r];
            double rhs = p3d_path_value(s, i, pn) - sig[i];
            for (int j = 0; j < 6; ++j)
                if (!(s->p3d_mask & (1 << j))) rhs -= D[i][j] * rate[j] * dt;
            for (int c = 0; c < m; ++c) A[r][c] = D[i][idx[c]];
            A[r][m] = rhs;
        }
        for (int c = 0; c < m; ++c) {          /* Gaussian elimination, partial pivoting */
            int piv = c;
            for (int r = c + 1; r < m; ++r) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
            for (int q = 0; q <= m; ++q) { double t = A[c][q]; A[c][q] = A[piv][q]; A[piv][q] = t; }
            for (int r = 0; r < m; ++r) {
                if (r == c) continue;
                const double f = A[r][c] / A[c][c];
                for (int q = c; q <= m; ++q) A[r][q] -= f * A[c][q];
            }
        }
        for (int r = 0; r < m; ++r) rate[idx[r]] = A[r][m] / A[r][r] / dt;
        s->p3d_first = 0;
    } else {
        /* later updates: the stress error extrapolated to the next step decides the
         * sign of a change of mod times the largest current rate */
        for (int i = 0; i < 6; ++i) {
            if (!(s->p3d_mask & (1 << i))) continue;
            const double pred = 2 * err[i] - s->p3d_err[i];
            if (pred > 0) rate[i] -= rmax * s->p3d_mod;
            else if (pred < 0) rate[i] += rmax * s->p3d_mod;
        }
    }
    for (int i = 0; i < 6; ++i) {
        if (rate[i] > s->p3d_max_rate) rate[i] = s->p3d_max_rate;
        if (rate[i] < -s->p3d_max_rate) rate[i] = -s->p3d_max_rate;
        s->p3d_rate[i] = rate[i];
        s->p3d_err[i] = err[i];
    }
    /* P+ = P + U^T (dt e_dot) U, T+ = U P+, grad(v) = (T+ T^-1 - I) / dt */
    double Ed[9] = {0}, A1[9], A2[9], Pn[9], Tn[9], Ti[9], L[9];
    for (int i = 0; i < 6; ++i) {
        const int a = VO[i][0], b = VO[i][1];
        if (a == b) Ed[3 * a + a] = dt * rate[i];
        else { Ed[3 * a + b] = 0.5 * dt * rate[i]; Ed[3 * b + a] = 0.5 * dt * rate[i]; }
    }
    m_mul(Ut, Ed, A1);
    m_mul(A1, U, A2);
    for (int q = 0; q < 9; ++q) Pn[q] = P[q] + A2[q];
    m_mul(U, Pn, Tn);
    m_inv(T, Ti);
    m_mul(Tn, Ti, L);
    for (int q = 0; q < 9; ++q) L[q] = (L[q] - (q % 4 == 0 ? 1.0 : 0.0)) / dt;
    memcpy(s->Lnext, L, sizeof L);
    s->L_pending = 1;
}

/* Peri3dController (class reference; reading R23).  goal, stress_mask (bit i: component
 * i of xx, yy, zz, yz, zx, xy is a stress), n_steps, mod, max_strain_rate,
 * young/poisson estimations, max_strain; paths: npath[i] couples (t, v) per component
 * (npath[i] = 0: the default linear path), at most 16; trsf0 (nullable: identity) the
 * cell transformation Cell.trsf already accumulated when the controller starts. */
int orc_set_peri3d(orc_scene *s, const double *goal, int stress_mask, long n_steps, double mod,
                   double max_strain_rate, double young_est, double poisson_est,
                   double max_strain, const int *npath, const double *path, const double *trsf0) {
    if (!s || !s->periodic || n_steps < 1 || !(max_strain_rate > 0) || !(young_est > 0) ||
        !(poisson_est > -1 && poisson_est < 0.5) || !(max_strain > 0) || !(mod >= 0))
        return -1;
    for (int i = 0; i < 6; ++i) {
        if (!isfinite(goal[i])) return -1;
        s->p3d_goal[i] = goal[i];
        const int n = npath ? npath[i] : 0;
        if (n < 0 || n > 16) return -1;
        if (n == 0) {
            s->p3d_npath[i] = 1;
            s->p3d_path[i][0][0] = 1; s->p3d_path[i][0][1] = 1;
        } else {
            s->p3d_npath[i] = n;
            for (int j = 0; j < n; ++j) {
                s->p3d_path[i][j][0] = path[(16 * i + j) * 2];
                s->p3d_path[i][j][1] = path[(16 * i + j) * 2 + 1];
            }
            if (!(s->p3d_path[i][n - 1][0] > 0) || s->p3d_path[i][n - 1][1] == 0) return -1;
            for (int j = 1; j < n; ++j) if (!(s->p3d_path[i][j][0] > s->p3d_path[i][j - 1][0])) return -1;
            if (!(s->p3d_path[i][0][0] > 0)) return -1;
        }
    }
    s->p3d = 1; s->triax = 0;
    s->p3d_mask = stress_mask & 63;
    s->p3d_nsteps = n_steps;
    s->p3d_mod = mod; s->p3d_max_rate = max_strain_rate;
    s->p3d_young = young_est; s->p3d_poisson = poisson_est; s->p3d_max_strain = max_strain;
    s->p3d_k = 0; s->p3d_first = 1; s->p3d_done = 0;
    memcpy(s->p3d_H0, s->H, sizeof s->H);
    for (int q = 0; q < 9; ++q) s->p3d_T0[q] = trsf0 ? trsf0[q] : (q % 4 == 0 ? 1.0 : 0.0);
    if (trsf0 && !(m_det(s->p3d_T0) > 0)) return -1;
    for (int i = 0; i < 6; ++i) { s->p3d_rate[i] = 0; s->p3d_err[i] = 0; s->p3d_stress[i] = 0; s->p3d_strain[i] = 0; }
    return 0;
}

/* stress[6], strain[6], rate[6] (nullable); returns 1 when done, 0 running, -1 off */
int orc_get_peri3d(const orc_scene *s, double *stress, double *strain, double *rate) {
    if (!s || !s->p3d) return -1;
    if (stress) memcpy(stress, s->p3d_stress, sizeof s->p3d_stress);
    if (strain) memcpy(strain, s->p3d_strain, sizeof s->p3d_strain);
    if (rate) memcpy(rate, s->p3d_rate, sizeof s->p3d_rate);
    return s->p3d_done;
}

int orc_set_triax(orc_scene *s, const double *goal, int stress_mask, const double *max_rate,
                  double grow_damping, int glob_update) {
    if (!s || !s->periodic || glob_update < 1 || !(grow_damping >= 0) || !(grow_damping < 1))
        return -1;
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(goal[a]) || !(max_rate[a] >= 0)) return -1;
        s->goal[a] = goal[a];
        s->max_rate[a] = max_rate[a];
    }
    s->stress_mask = stress_mask & 7;
    s->grow_damping = grow_damping;
    s->glob_update = glob_update;
    s->triax = 1;
    s->p3d = 0;
    return 0;
}

/* GlobalStiffnessTimeStepper (section 2.1.5 "Stability considerations", eq. 2.12-2.14,
 * GlobalStiffnessTimeStepper class reference; reading R17).  Per body, the diagonal of
 * its translational stiffness K_ii = sum over its contacts of (kn - ks) n_i^2 + ks
 * (eq. 2.14) and of its rotational stiffness sum ks d^2 (1 - n_i^2) (the shear spring
 * at the arm d = r - pen/2 from the centre); per degree of freedom the critical step
 * sqrt(2) sqrt(m / K) (eq. 2.12, DOFs taken as uncoupled as the text prescribes); the
 * time step is the safety coefficient times the smallest of them over the free
 * bodies, or, when no body has a contact, defaultDt (or the safety coefficient times
 * the p-wave step when defaultDt < 0); capped by maxDt when that is positive. */
static void stiffness_dt(orc_scene *s) {
    long n = s->n;
    double *Kt = (double *)calloc(3 * (size_t)n + 1, sizeof(double));
    double *Kr = (double *)calloc(3 * (size_t)n + 1, sizeof(double));
    if (!Kt || !Kr) { free(Kt); free(Kr); return; }
    for (long k = 0; k < s->ncon; ++k) {
        const orc_contact *ct = &s->con[k];
        long bodies[2] = {ct->id1, ct->id2};
        double kn, ks;
        tangent_stiffness(s, ct, &kn, &ks);
        for (int e = 0; e < 2; ++e) {
            long b = bodies[e];
            if (b < 0) continue;   /* the wall side */
            double d = s->radius[b] - 0.5 * ct->pen;
            for (int i = 0; i < 3; ++i) {
                double ni2 = ct->n[i] * ct->n[i];
                Kt[3 * b + i] += (kn - ks) * ni2 + ks;
                Kr[3 * b + i] += ks * d * d * (1.0 - ni2);
            }
        }
    }
    double best = INFINITY;
    for (long b = 0; b < n; ++b) {
        if (s->fixed[b]) continue;
        double tb = INFINITY;   /* this body's critical step (eq. 2.12, unscaled masses) */
        for (int i = 0; i < 3; ++i) {
            if (Kt[3 * b + i] > 0) {
                double t = sqrt(2.0) * sqrt(s->mass[b] / Kt[3 * b + i]);
                if (t < tb) tb = t;
            }
            if (Kr[3 * b + i] > 0) {
                double t = sqrt(2.0) * sqrt(s->inertia[b] / Kr[3 * b + i]);
                if (t < tb) tb = t;
            }
        }
        if (tb < best) best = tb;
        /* density scaling (R22): inertia scaled by f so that safety * sqrt(f) * tb is the
         * target step; a body without contacts keeps its factor */
        if (s->dscale_on && !isinf(tb)) {
            double ratio = s->target_dt / (s->tstep_safety * tb);
            s->dscale[b] = ratio * ratio;
        }
    }
    free(Kt);
    free(Kr);
    if (s->dscale_on) { s->dt = s->target_dt; return; }
    double dt;
    if (isinf(best)) dt = s->tstep_default > 0 ? s->tstep_default : s->tstep_safety * orc_pwave_dt(s);
    else dt = s->tstep_safety * best;
    if (s->tstep_max > 0 && dt > s->tstep_max) dt = s->tstep_max;
    s->dt = dt;
}

/* NewtonIntegrator.densityScaling with GlobalStiffnessTimeStepper.targetDt (reading
 * R22): needs the time stepper; on each stepper update every free body with contacts
 * gets the inertia factor f = (target_dt / (safety * t_b))^2, t_b its critical step
 * of eq. 2.12, and the step becomes target_dt.  Turning it off restores f = 1. */
int orc_set_density_scaling(orc_scene *s, int on, double target_dt) {
    if (!s) return -1;
    if (on && (!s->tstep || !(target_dt > 0) || !isfinite(target_dt))) return -1;
    s->dscale_on = on ? 1 : 0;
    s->target_dt = on ? target_dt : 0.0;
    if (!on)
        for (long i = 0; i < s->n; ++i) s->dscale[i] = 1.0;
    return 0;
}

void orc_get_density_scaling(const orc_scene *s, double *f) {
    if (f) memcpy(f, s->dscale, sizeof(double) * s->n);
}

int orc_set_timestepper(orc_scene *s, double safety, int interval, double default_dt,
                        double max_dt) {
    if (!s || !(safety > 0) || interval < 1 || !isfinite(default_dt) || !isfinite(max_dt)) return -1;
    s->tstep = 1;
    s->tstep_safety = safety;
    s->tstep_interval = interval;
    s->tstep_default = default_dt;
    s->tstep_max = max_dt;
    return 0;
}

static int step_once(orc_scene *s) {
    const double dt = s->dt;
    if (!(dt > 0)) return -1;
    if (s->L_pending) { memcpy(s->L, s->Lnext, sizeof s->L); s->L_pending = 0; }
    int rc = check_cell(s);
    if (rc) return rc;
    /* ForceResetter */
    memset(s->force, 0, sizeof(double) * 3 * s->n);
    memset(s->torque, 0, sizeof(double) * 3 * s->n);
    /* collider */
    orc_contact *nc = NULL;
    long nn = 0;
    rc = detect_contacts(s, &nc, &nn);
    if (rc) return rc;
    free(s->con);
    s->con = nc;
    s->ncon = nn;
    s->capcon = nn;
    /* image velocity of body 2: v2 + grad(v)_prev H_prev c (R8) */
    double W[9];
    m_mul(s->Lprev, s->Hprev, W);
    /* InteractionLoop: Ig2 -> Ip2 (new) -> Law2, forces applied to both bodies */
    for (long k = 0; k < s->ncon; ++k) {
        orc_contact *ct = &s->con[k];
        double F2[3], F1[3], T[3], arm[3];
        if (ct->id1 < 0) {
            /* Ig2_Wall_Sphere_ScGeom (R10) */
            int w = -ct->id1 - 1, ax = w >> 1;
            long j = ct->id2;
            const double *x2 = s->pos + 3 * j;
            double r = s->radius[j];
            double dist = x2[ax] - wall_coord(s, w);
            double n[3] = {0, 0, 0};
            n[ax] = dist >= 0 ? 1.0 : -1.0;
            double pen = r - fabs(dist);
            if (ct->kn == 0) {
                if (s->law == 1)
                    ip2_mindlin(&s->mats[s->mat[j]], r, &s->mats[0], -1.0, &ct->kn, &ct->ks,
                                &ct->tanphi);
                else
                    ip2_frict(&s->mats[0], r, &s->mats[s->mat[j]], r, &ct->kn, &ct->ks, &ct->tanphi);
                for (int q = 0; q < 3; ++q) { ct->nprev[q] = n[q]; ct->fs[q] = 0; }
            }
            double zero[3] = {0, 0, 0};
            shear_and_law(ct, n, pen, zero, zero, s->vel + 3 * j, s->angvel + 3 * j, r, r,
                          2 * r - pen, dt, s->law, F2, &s->plast_dissip);
            for (int q = 0; q < 3; ++q) ct->cp[q] = x2[q] - (r - 0.5 * pen) * n[q];
            for (int q = 0; q < 3; ++q) arm[q] = ct->cp[q] - x2[q];
            v_cross(arm, F2, T);
            for (int q = 0; q < 3; ++q) { s->force[3 * j + q] += F2[q]; s->torque[3 * j + q] += T[q]; }
            continue;
        }
        long i = ct->id1, j = ct->id2;
        const double *x1 = s->pos + 3 * i, *x2 = s->pos + 3 * j;
        double r1 = s->radius[i], r2 = s->radius[j];
        double h[3] = {0, 0, 0}, d[3], x2i[3], v2i[3], wc[3];
        if (s->periodic) cell_shift(s->H, ct->c, h);
        double d2 = branch(x1, x2, h, d);
        double l = sqrt(d2);
        double n[3] = {d[0] / l, d[1] / l, d[2] / l};              /* eq. 2.7 */
        double pen = (r1 + r2) - l;                                 /* penetrationDepth */
        for (int q = 0; q < 3; ++q) x2i[q] = x2[q] + h[q];
        double cd[3] = {(double)ct->c[0], (double)ct->c[1], (double)ct->c[2]};
        m_vec(W, cd, wc);
        for (int q = 0; q < 3; ++q) v2i[q] = s->vel[3 * j + q] + (s->periodic ? wc[q] : 0.0);
        if (ct->kn == 0) {
            if (s->law == 1)
                ip2_mindlin(&s->mats[s->mat[i]], r1, &s->mats[s->mat[j]], r2, &ct->kn, &ct->ks,
                            &ct->tanphi);
            else
                ip2_frict(&s->mats[s->mat[i]], r1, &s->mats[s->mat[j]], r2, &ct->kn, &ct->ks,
                          &ct->tanphi);
            for (int q = 0; q < 3; ++q) { ct->nprev[q] = n[q]; ct->fs[q] = 0; }   /* R6 */
        }
        shear_and_law(ct, n, pen, s->vel + 3 * i, s->angvel + 3 * i, v2i, s->angvel + 3 * j,
                      r1, r2, l, dt, s->law, F2, &s->plast_dissip);
        for (int q = 0; q < 3; ++q) { ct->cp[q] = x1[q] + (r1 - 0.5 * pen) * n[q]; F1[q] = -F2[q]; }
        /* torques from the contact point (R4) */
        for (int q = 0; q < 3; ++q) arm[q] = ct->cp[q] - x1[q];
        v_cross(arm, F1, T);
        for (int q = 0; q < 3; ++q) { s->force[3 * i + q] += F1[q]; s->torque[3 * i + q] += T[q]; }
        for (int q = 0; q < 3; ++q) arm[q] = ct->cp[q] - x2i[q];
        v_cross(arm, F2, T);
        for (int q = 0; q < 3; ++q) { s->force[3 * j + q] += F2[q]; s->torque[3 * j + q] += T[q]; }
    }
    /* GlobalStiffnessTimeStepper between InteractionLoop and NewtonIntegrator (the
     * engine order of the text's scripts): the new step integrates this step */
    if (s->tstep && s->iter % s->tstep_interval == 0) stiffness_dt(s);
    const double dtN = s->dt;
    /* NewtonIntegrator */
    const double lam = s->damping;
    double dL[9];
    for (int q = 0; q < 9; ++q) dL[q] = s->L[q] - s->Lprev[q];
    for (long i = 0; i < s->n; ++i) {
        double *x = s->pos + 3 * i, *v = s->vel + 3 * i, *w = s->angvel + 3 * i;
        /* inertial mass and moment: scaled by the density-scaling factor (R22, 1 when
         * off); the weight stays the true m g */
        double m = s->mass[i] * s->dscale[i], I = s->inertia[i] * s->dscale[i];
        double vold[3] = {v[0], v[1], v[2]}, xold[3] = {x[0], x[1], x[2]};
        if (!s->fixed[i]) {
            double F[3], T[3], vref[3];
            for (int q = 0; q < 3; ++q) {
                F[q] = s->force[3 * i + q] + s->mass[i] * s->g[q];
                T[q] = s->torque[3 * i + q];
            }
            /* eq. 2.9 velocity: fluctuation part in a periodic cell (R7) */
            if (s->periodic) {
                double mf[3];
                m_vec(s->Lprev, xold, mf);
                for (int q = 0; q < 3; ++q) vref[q] = vold[q] - mf[q];
            } else {
                for (int q = 0; q < 3; ++q) vref[q] = vold[q];
            }
            double Fd[3], Td[3];
            for (int q = 0; q < 3; ++q) {
                double acc = F[q] / m;
                Fd[q] = F[q] * (1 - lam * sgn(F[q] * (vref[q] + 0.5 * dtN * acc)));
                double aacc = T[q] / I;
                Td[q] = T[q] * (1 - lam * sgn(T[q] * (w[q] + 0.5 * dtN * aacc)));
            }
            /* leapfrog: v+ = v- + dt F/m ; w+ = w- + dt T/I */
            for (int q = 0; q < 3; ++q) {
                v[q] = vold[q] + dtN * Fd[q] / m;
                w[q] = w[q] + dtN * Td[q] / I;
            }
            if (s->periodic) {
                /* homoDeform = 2 (R9): (grad(v) - grad(v)_prev) x + dt grad(v) v- */
                double a1[3], a2[3];
                m_vec(dL, xold, a1);
                m_vec(s->L, vold, a2);
                for (int q = 0; q < 3; ++q) v[q] = v[q] + a1[q] + dtN * a2[q];
            }
            /* energy tracker: damping work, gravity work (sign conventions of the doctest
             * in the yade.plot reference) */
            for (int q = 0; q < 3; ++q) {
                s->nonvisc_damp += -(Fd[q] - F[q]) * v[q] * dtN;
                s->nonvisc_damp += -(Td[q] - T[q]) * w[q] * dtN;
                s->grav_work += -s->mass[i] * s->g[q] * v[q] * dtN;
            }
        }
        for (int q = 0; q < 3; ++q) x[q] = xold[q] + dtN * v[q];
        /* orientation: q+ = dq(w+ dt) q (spherical rotation, section 2.1.5) */
        double wn = sqrt(v_dot(w, w));
        if (wn > 0) {
            double ang = wn * dtN;
            double sh = sin(0.5 * ang), ch = cos(0.5 * ang);
            double dq[4] = {ch, sh * w[0] / wn, sh * w[1] / wn, sh * w[2] / wn};
            quat_mul(dq, s->ori + 4 * i, s->ori + 4 * i);
        }
    }
    /* cell: H+ = (I + grad(v) dt) H (section 2.1.6) */
    if (s->periodic) {
        double A[9];
        for (int q = 0; q < 9; ++q) A[q] = (q % 4 == 0 ? 1.0 : 0.0) + s->L[q] * dtN;
        memcpy(s->Hprev, s->H, sizeof s->H);
        m_mul(A, s->H, s->H);
        memcpy(s->Lprev, s->L, sizeof s->L);
    }
    s->time += dtN;
    s->iter += 1;
    if (s->triax && s->periodic && s->iter % s->glob_update == 0) triax_update(s);
    if (s->p3d && s->periodic) p3d_update(s);
    return 0;
}

int orc_step(orc_scene *s, long nsteps) {
    if (!s || nsteps < 0) return -1;
    for (long k = 0; k < nsteps; ++k) {
        int rc = step_once(s);
        if (rc) return rc;
    }
    return 0;
}

long orc_num_bodies(const orc_scene *s) { return s ? s->n : 0; }

void orc_get_state(const orc_scene *s, double *pos, double *vel, double *angvel, double *ori,
                   double *force, double *torque) {
    if (pos) memcpy(pos, s->pos, sizeof(double) * 3 * s->n);
    if (vel) memcpy(vel, s->vel, sizeof(double) * 3 * s->n);
    if (angvel) memcpy(angvel, s->angvel, sizeof(double) * 3 * s->n);
    if (ori) memcpy(ori, s->ori, sizeof(double) * 4 * s->n);
    if (force) memcpy(force, s->force, sizeof(double) * 3 * s->n);
    if (torque) memcpy(torque, s->torque, sizeof(double) * 3 * s->n);
}

int orc_set_state(orc_scene *s, const double *pos, const double *vel, const double *angvel,
                  const double *ori) {
    if (!s) return -1;
    if (pos) memcpy(s->pos, pos, sizeof(double) * 3 * s->n);
    if (vel) memcpy(s->vel, vel, sizeof(double) * 3 * s->n);
    if (angvel) memcpy(s->angvel, angvel, sizeof(double) * 3 * s->n);
    if (ori) memcpy(s->ori, ori, sizeof(double) * 4 * s->n);
    return 0;
}

void orc_get_cell(const orc_scene *s, double *H9, double *velgrad9, double *prev_velgrad9,
                  double *prev_H9) {
    if (H9) memcpy(H9, s->H, sizeof s->H);
    if (velgrad9) memcpy(velgrad9, s->L_pending ? s->Lnext : s->L, sizeof s->L);
    if (prev_velgrad9) memcpy(prev_velgrad9, s->Lprev, sizeof s->Lprev);
    if (prev_H9) memcpy(prev_H9, s->Hprev, sizeof s->Hprev);
}

int orc_set_cell(orc_scene *s, const double *H9, const double *velgrad9,
                 const double *prev_velgrad9, const double *prev_H9) {
    if (!s || !s->periodic) return -1;
    if (H9) memcpy(s->H, H9, sizeof s->H);
    if (velgrad9) { memcpy(s->L, velgrad9, sizeof s->L); s->L_pending = 0; }
    if (prev_velgrad9) memcpy(s->Lprev, prev_velgrad9, sizeof s->Lprev);
    if (prev_H9) memcpy(s->Hprev, prev_H9, sizeof s->Hprev);
    return 0;
}

/* utils.flipCell (section 2.1.6, "Collision detection in periodic cell", fig. 6): the
 * corners of the periodic cell repeated in space form a lattice, and any other cell
 * spanning the same lattice describes the same periodic space.  The new cell is
 * H' = H M with M = I + K an integer matrix of determinant 1; positions do not move,
 * and each interaction keeps its image: x2 + H c = x2 + H' c' with c' = M^-1 c.
 * The image-velocity matrix Hprev changes the same way (Lprev Hprev c is invariant).
 * K given: used as is (rejected unless det(I + K) = 1 and the new diagonal is
 * positive).  K NULL: the automatic reduction of reading R21, one pass over the
 * column pairs (i, j) in the order (1,2) (0,2) (0,1) (1,0) (2,0) (2,1): with
 * k = round(H_ij / H_ii), column j -= k * column i, skipped when k = 0 or when it
 * would make H_jj non-positive.  The applied K is written to `applied` (nullable).
 * Returns 0, or -1 (aperiodic scene, invalid K, or a shift out of range). */
int orc_flip_cell(orc_scene *s, const int *K9, int *applied) {
    if (!s || !s->periodic) return -1;
    int M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (K9) {
        for (int q = 0; q < 9; ++q) M[q] += K9[q];
    } else {
        double Hc[9];
        memcpy(Hc, s->H, sizeof Hc);
        static const int order[6][2] = {{1, 2}, {0, 2}, {0, 1}, {1, 0}, {2, 0}, {2, 1}};
        for (int p = 0; p < 6; ++p) {
            const int i = order[p][0], j = order[p][1];
            const double k = floor(Hc[3 * i + j] / Hc[3 * i + i] + 0.5);
            if (k == 0 || !(Hc[3 * j + j] - k * Hc[3 * j + i] > 0)) continue;
            /* column j of H and of M lose k times column i */
            for (int r = 0; r < 3; ++r) {
                Hc[3 * r + j] -= k * Hc[3 * r + i];
                M[3 * r + j] -= (int)k * M[3 * r + i];
            }
        }
    }
    /* integer inverse by the adjugate (det M = 1) */
    const long det = (long)M[0] * (M[4] * M[8] - M[5] * M[7]) - (long)M[1] * (M[3] * M[8] - M[5] * M[6]) +
                     (long)M[2] * (M[3] * M[7] - M[4] * M[6]);
    if (det != 1) return -1;
    int Mi[9];
    Mi[0] = M[4] * M[8] - M[5] * M[7]; Mi[1] = M[2] * M[7] - M[1] * M[8]; Mi[2] = M[1] * M[5] - M[2] * M[4];
    Mi[3] = M[5] * M[6] - M[3] * M[8]; Mi[4] = M[0] * M[8] - M[2] * M[6]; Mi[5] = M[2] * M[3] - M[0] * M[5];
    Mi[6] = M[3] * M[7] - M[4] * M[6]; Mi[7] = M[1] * M[6] - M[0] * M[7]; Mi[8] = M[0] * M[4] - M[1] * M[3];
    double Md[9], Hn[9], Hpn[9];
    for (int q = 0; q < 9; ++q) Md[q] = (double)M[q];
    m_mul(s->H, Md, Hn);
    m_mul(s->Hprev, Md, Hpn);
    if (!(Hn[0] > 0 && Hn[4] > 0 && Hn[8] > 0)) return -1;
    for (long k = 0; k < s->ncon; ++k) {
        const int *c = s->con[k].c;
        for (int r = 0; r < 3; ++r) {
            const long v = (long)Mi[3 * r] * c[0] + (long)Mi[3 * r + 1] * c[1] + (long)Mi[3 * r + 2] * c[2];
            if (v > 511 || v < -511) return -1;   /* the library's shift range */
        }
    }
    for (long k = 0; k < s->ncon; ++k) {
        int *c = s->con[k].c, o[3];
        for (int r = 0; r < 3; ++r) o[r] = Mi[3 * r] * c[0] + Mi[3 * r + 1] * c[1] + Mi[3 * r + 2] * c[2];
        c[0] = o[0]; c[1] = o[1]; c[2] = o[2];
    }
    memcpy(s->H, Hn, sizeof Hn);
    memcpy(s->Hprev, Hpn, sizeof Hpn);
    if (applied)
        for (int q = 0; q < 9; ++q) applied[q] = M[q] - ((q % 4 == 0) ? 1 : 0);
    return 0;
}

void orc_get_clock(const orc_scene *s, long *iter, double *time, double *dt) {
    if (iter) *iter = s->iter;
    if (time) *time = s->time;
    if (dt) *dt = s->dt;
}

int orc_set_clock(orc_scene *s, long iter, double time) {
    if (!s || iter < 0) return -1;
    s->iter = iter;
    s->time = time;
    return 0;
}

long orc_num_contacts(const orc_scene *s) { return s ? s->ncon : 0; }

long orc_get_contacts(const orc_scene *s, long cap, int *id1, int *id2, int *c, double *fn,
                      double *fs, double *normal, double *cpoint, double *phys, double *pen) {
    long m = s->ncon < cap ? s->ncon : cap;
    for (long k = 0; k < m; ++k) {
        const orc_contact *ct = &s->con[k];
        if (id1) id1[k] = ct->id1;
        if (id2) id2[k] = ct->id2;
        for (int q = 0; q < 3; ++q) {
            if (c) c[3 * k + q] = ct->c[q];
            if (fn) fn[3 * k + q] = ct->fn * ct->n[q];
            if (fs) fs[3 * k + q] = ct->fs[q];
            if (normal) normal[3 * k + q] = ct->n[q];
            if (cpoint) cpoint[3 * k + q] = ct->cp[q];
        }
        if (phys) { phys[3 * k] = ct->kn; phys[3 * k + 1] = ct->ks; phys[3 * k + 2] = ct->tanphi; }
        if (pen) pen[k] = ct->pen;
    }
    return m;
}

int orc_set_contacts(orc_scene *s, long n, const int *id1, const int *id2, const int *c,
                     const double *fs, const double *nprev, const double *phys) {
    if (!s || n < 0) return -1;
    orc_contact *nc = (orc_contact *)calloc(n + 1, sizeof(orc_contact));
    if (!nc) return -2;
    for (long k = 0; k < n; ++k) {
        orc_contact *ct = &nc[k];
        ct->id1 = id1[k]; ct->id2 = id2[k];
        if (ct->id2 < 0 || ct->id2 >= s->n || ct->id1 >= ct->id2 || ct->id1 < -6) { free(nc); return -1; }
        if (k > 0 && (nc[k - 1].id1 > ct->id1 || (nc[k - 1].id1 == ct->id1 && nc[k - 1].id2 >= ct->id2))) {
            free(nc); return -1; /* rows must be sorted by (id1, id2) without repeats */
        }
        for (int q = 0; q < 3; ++q) {
            ct->c[q] = c ? c[3 * k + q] : 0;
            ct->fs[q] = fs[3 * k + q];
            ct->nprev[q] = nprev[3 * k + q];
            ct->n[q] = nprev[3 * k + q];
        }
        ct->kn = phys[3 * k]; ct->ks = phys[3 * k + 1]; ct->tanphi = phys[3 * k + 2];
    }
    free(s->con);
    s->con = nc;
    s->ncon = n;
    s->capcon = n;
    return 0;
}

void orc_get_energy(const orc_scene *s, double *out) {
    double kt = 0, kr = 0, el = 0;
    for (long i = 0; i < s->n; ++i) {
        const double *v = s->vel + 3 * i, *w = s->angvel + 3 * i;
        kt += 0.5 * s->mass[i] * v_dot(v, v);
        kr += 0.5 * s->inertia[i] * v_dot(w, w);
    }
    for (long k = 0; k < s->ncon; ++k) {
        const orc_contact *ct = &s->con[k];
        double kn, ks;
        tangent_stiffness(s, ct, &kn, &ks);
        /* normal spring energy: Fn^2 / (2 kn) (linear), 2/5 kno pen^5/2 = 2/5 Fn pen (Hertz) */
        if (s->law == 1) el += 0.4 * ct->fn * ct->pen;
        else if (kn > 0) el += ct->fn * ct->fn / (2 * kn);
        if (ks > 0) el += v_dot(ct->fs, ct->fs) / (2 * ks);
    }
    out[0] = kt; out[1] = kr; out[2] = s->grav_work; out[3] = s->nonvisc_damp;
    out[4] = s->plast_dissip; out[5] = el;
    out[6] = kt + kr + s->grav_work + s->nonvisc_damp + s->plast_dissip + el;
}

void orc_get_stats(const orc_scene *s, double *out) {
    /* kinetic energy (utils.kineticEnergy): sum of 1/2 (m v^2 + I w^2) */
    double ke = 0;
    long ndyn = 0;
    double sumF = 0;
    for (long i = 0; i < s->n; ++i) {
        const double *v = s->vel + 3 * i, *w = s->angvel + 3 * i;
        ke += 0.5 * s->mass[i] * v_dot(v, v) + 0.5 * s->inertia[i] * v_dot(w, w);
        if (!s->fixed[i]) { ++ndyn; sumF += sqrt(v_dot(s->force + 3 * i, s->force + 3 * i)); }
    }
    /* unbalanced force: mean body contact force / mean contact force */
    double sumC = 0;
    long nc = 0, nss = 0;
    double sig[9] = {0};
    for (long k = 0; k < s->ncon; ++k) {
        const orc_contact *ct = &s->con[k];
        double F2[3];
        for (int q = 0; q < 3; ++q) F2[q] = ct->fn * ct->n[q] + ct->fs[q];
        sumC += sqrt(v_dot(F2, F2));
        ++nc;
        if (ct->id1 >= 0) {
            ++nss;
            /* Love-Weber stress: (1/V) sum f_i l_j with f on body 2, l = x1 - x2' */
            double l = (s->radius[ct->id1] + s->radius[ct->id2]) - ct->pen;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) sig[3 * a + b] += F2[a] * (-l * ct->n[b]);
        }
    }
    double V;
    if (s->periodic) V = fabs(m_det(s->H));
    else V = (s->box_hi[0] - s->box_lo[0]) * (s->box_hi[1] - s->box_lo[1]) * (s->box_hi[2] - s->box_lo[2]);
    double vs = 0;
    for (long i = 0; i < s->n; ++i) vs += (4.0 / 3.0) * 3.14159265358979323846 * s->radius[i] * s->radius[i] * s->radius[i];
    out[0] = ke;
    out[1] = (nc > 0 && ndyn > 0) ? (sumF / ndyn) / (sumC / nc) : NAN;
    out[2] = s->n > 0 ? 2.0 * nss / s->n : 0;
    out[3] = vs / V;
    out[4] = (double)nss;
    for (int q = 0; q < 9; ++q) out[5 + q] = sig[q] / V;
}
