/*
 * Seeded random sequential placement of non-overlapping spheres.
 *
 * Input generation only: this file holds none of the DEM method's arithmetic.
 * It plays the role of the loose-cloud generator of the Yade text
 * (SpherePack.makeCloud, section "yade.pack"): every sphere draws uniform
 * random centres until it overlaps no sphere placed before it.  Spheres are
 * placed in descending radius order (large first) so that dense-ish clouds
 * (solid fraction 0.3) are reachable; the position is written back to the
 * sphere's original index, so ids stay uncorrelated with size.
 *
 * The random stream is splitmix64 (Steele, Lea & Flood 2014), so the same
 * seed gives the same cloud on every platform (no libm call on the path that
 * decides an overlap; build with -ffp-contract=off).
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>

static uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double sm64_unit(uint64_t *s) { /* [0,1) with 53 random bits */
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

/* Fill out[0..n) with uniform [0,1) numbers from splitmix64(seed). */
void wl_uniform(long n, uint64_t seed, double *out) {
    uint64_t s = seed;
    for (long i = 0; i < n; ++i) out[i] = sm64_unit(&s);
}

typedef struct { long idx; double r; } rsa_item;

static int cmp_desc(const void *a, const void *b) {
    const rsa_item *x = (const rsa_item *)a, *y = (const rsa_item *)b;
    if (x->r > y->r) return -1;
    if (x->r < y->r) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/*
 * Place n spheres.  Aperiodic: centres in [lo+r, hi-r] per axis.  Periodic:
 * centres in [lo, hi) with minimum-image overlap tests (cell edge hi-lo).
 * Returns 0 on success, -1 on allocation failure, -2 when a sphere found no
 * free spot within max_attempts draws, -3 on bad arguments.
 */
int wl_rsa_place(long n, const double *radius, const double *lo, const double *hi,
                 int periodic, uint64_t seed, long max_attempts, double *pos) {
    if (n <= 0) return 0;
    double rmax = 0;
    for (long i = 0; i < n; ++i) {
        if (!(radius[i] > 0)) return -3;
        if (radius[i] > rmax) rmax = radius[i];
    }
    double ext[3];
    int nc[3];
    double cs[3];
    for (int k = 0; k < 3; ++k) {
        ext[k] = hi[k] - lo[k];
        if (!(ext[k] > 0)) return -3;
        if (!periodic && ext[k] < 2 * rmax) return -3;
        nc[k] = (int)floor(ext[k] / (2.0 * rmax));
        if (nc[k] < 1) nc[k] = 1;
        if (nc[k] > 1024) nc[k] = 1024;
        cs[k] = ext[k] / nc[k];
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    long *head = (long *)malloc(sizeof(long) * ncell);
    long *next = (long *)malloc(sizeof(long) * n);
    rsa_item *order = (rsa_item *)malloc(sizeof(rsa_item) * n);
    if (!head || !next || !order) { free(head); free(next); free(order); return -1; }
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (long i = 0; i < n; ++i) { order[i].idx = i; order[i].r = radius[i]; }
    qsort(order, n, sizeof(rsa_item), cmp_desc);

    uint64_t st = seed;
    int rc = 0;
    for (long t = 0; t < n && rc == 0; ++t) {
        long i = order[t].idx;
        double ri = radius[i];
        int placed = 0;
        for (long att = 0; att < max_attempts && !placed; ++att) {
            double p[3];
            for (int k = 0; k < 3; ++k) {
                double u = sm64_unit(&st);
                if (periodic) p[k] = lo[k] + u * ext[k];
                else p[k] = (lo[k] + ri) + u * (ext[k] - 2 * ri);
            }
            int ci[3];
            for (int k = 0; k < 3; ++k) {
                int c = (int)floor((p[k] - lo[k]) / cs[k]);
                if (c < 0) c = 0;
                if (c >= nc[k]) c = nc[k] - 1;
                ci[k] = c;
            }
            int ok = 1;
            /* distinct neighbour cells per axis (a wrap with nc<3 would repeat a cell) */
            int nb[3][3], nnb[3];
            for (int k = 0; k < 3; ++k) {
                nnb[k] = 0;
                for (int d = -1; d <= 1; ++d) {
                    int c = ci[k] + d;
                    if (periodic) { c %= nc[k]; if (c < 0) c += nc[k]; }
                    else if (c < 0 || c >= nc[k]) continue;
                    int dup = 0;
                    for (int q = 0; q < nnb[k]; ++q) if (nb[k][q] == c) dup = 1;
                    if (!dup) nb[k][nnb[k]++] = c;
                }
            }
            for (int a = 0; a < nnb[0] && ok; ++a)
                for (int b = 0; b < nnb[1] && ok; ++b)
                    for (int c = 0; c < nnb[2] && ok; ++c) {
                        long cell = ((long)nb[0][a] * nc[1] + nb[1][b]) * nc[2] + nb[2][c];
                        for (long j = head[cell]; j >= 0; j = next[j]) {
                            double d2 = 0;
                            for (int k = 0; k < 3; ++k) {
                                double d = pos[3 * j + k] - p[k];
                                if (periodic) {
                                    if (d > 0.5 * ext[k]) d -= ext[k];
                                    else if (d < -0.5 * ext[k]) d += ext[k];
                                }
                                d2 += d * d;
                            }
                            double rs = radius[j] + ri;
                            if (d2 < rs * rs) { ok = 0; break; }
                        }
                    }
            if (ok) {
                for (int k = 0; k < 3; ++k) pos[3 * i + k] = p[k];
                long cell = ((long)ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
                next[i] = head[cell];
                head[cell] = i;
                placed = 1;
            }
        }
        if (!placed) rc = -2;
    }
    free(head); free(next); free(order);
    return rc;
}
