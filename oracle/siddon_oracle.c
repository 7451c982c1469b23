/*
 * FP64 reference projector for BSGD -- TEST INFRASTRUCTURE ONLY.
 *
 * Part of the oracle: plain, slow, obviously correct CPU code that the tests,
 * the smoke check and the CPU-baseline leg of bench.py use to check the CUDA
 * library. The library never links, loads or calls anything in oracle/.
 *
 * What it computes (Sec. 1, Eq. 1 and the paragraph after it): y = A x with
 * A_{ij} >= 0 the length of ray i inside voxel j, the entries that Siddon's
 * method produces. The traversal below is the original plane-crossing form of
 * Siddon's algorithm, written from its definition:
 *
 *   1. the ray is p(a) = p0 + a (p1 - p0), a in [0, 1];
 *   2. clip it to the volume box: [a_min, a_max];
 *   3. collect the parameters a at which it crosses every grid plane strictly
 *      inside (a_min, a_max), add a_min and a_max, and sort them;
 *   4. each interval [a_k, a_{k+1}] of positive width lies in exactly one voxel,
 *      the one containing its midpoint; its length is (a_{k+1} - a_k) |p1 - p0|.
 *
 * A column block J (Sec. 2, Eq. 3) is a slab of whole voxel planes along the
 * block axis (z for 3D volumes, y for 2D images); A_I^J keeps the segments whose
 * voxel lies in that slab, which is the sub-matrix definition itself.
 *
 * Geometry conventions (the paper fixes none; these are the readings used on
 * both sides of the parity tests):
 *   - volume [z][y][x], x fastest; voxel i along an axis with n voxels of size h
 *     spans [-n h / 2 + i h, -n h / 2 + (i + 1) h];
 *   - sinogram [view][v][u], u fastest; pixel centre (k - (n - 1) / 2) * size;
 *   - parallel 2D: direction (cos t, sin t, 0), detector axis (-sin t, cos t, 0);
 *   - fan 2D / cone 3D: source dso (cos b, sin b, 0), detector centre
 *     -(dsd - dso)(cos b, sin b, 0), axes u = (-sin b, cos b, 0), v = (0, 0, 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int kind;             /* 0 parallel 2D, 1 fan 2D, 2 cone 3D */
    int nx, ny, nz;
    double dx, dy, dz;
    int n_views;
    const double *angles; /* n_views view angles, radians */
    int nu, nv;
    double du, dv;
    double dso, dsd;
} orc_geom;

/* cos and sin of a view angle. An angle within 1e-9 rad of a multiple of
 * pi / 2 is that multiple exactly: its directions are axis-aligned, so a ray
 * of such a view that lies in a voxel face lies exactly in it (double cos(pi/2)
 * is 6e-17, a tilt that would decide, for a ray in a face, which of the two
 * voxel columns receives the whole ray). */
static void orc_cos_sin(double t, double *c, double *s)
{
    const double quarter = 1.5707963267948966; /* pi / 2 */
    const double k = nearbyint(t / quarter);
    if (fabs(t - k * quarter) <= 1e-9) {
        const long long m = (((long long)k % 4) + 4) % 4;
        *c = m == 0 ? 1.0 : (m == 2 ? -1.0 : 0.0);
        *s = m == 1 ? 1.0 : (m == 3 ? -1.0 : 0.0);
        return;
    }
    *c = cos(t);
    *s = sin(t);
}

/* End points p0, p1 of the ray of pixel (u, v) at view a. */
static void orc_ray(const orc_geom *g, int a, int v, int u, double p0[3], double p1[3])
{
    double c, s;
    orc_cos_sin(g->angles[a], &c, &s);
    double uc = (u - 0.5 * (g->nu - 1)) * g->du;
    double vc = (v - 0.5 * (g->nv - 1)) * g->dv;
    if (g->kind == 0) {
        /* parallel beam: a segment through the bin centre along (c, s), long
           enough to cross the whole volume box */
        double hx = 0.5 * g->nx * g->dx, hy = 0.5 * g->ny * g->dy, hz = 0.5 * g->nz * g->dz;
        double R = sqrt(hx * hx + hy * hy + hz * hz) + 1.0;
        double bx = -s * uc, by = c * uc;
        p0[0] = bx - R * c; p0[1] = by - R * s; p0[2] = 0.0;
        p1[0] = bx + R * c; p1[1] = by + R * s; p1[2] = 0.0;
    } else {
        double back = g->dsd - g->dso;
        p0[0] = g->dso * c; p0[1] = g->dso * s; p0[2] = 0.0;
        p1[0] = -back * c - s * uc;
        p1[1] = -back * s + c * uc;
        p1[2] = vc;
    }
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Largest number of segments one ray can produce (plus the two end points). */
static int orc_max_crossings(const orc_geom *g) { return g->nx + g->ny + g->nz + 8; }

/*
 * Siddon traversal of segment p0 -> p1 through the whole volume.
 * Writes the flat voxel index and the length of every interval of positive
 * length; returns their number. `alpha` is scratch of orc_max_crossings() doubles.
 */
static int orc_trace(const orc_geom *g, const double p0[3], const double p1[3],
                     int64_t *vox, double *len, double *alpha)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const double h[3] = {g->dx, g->dy, g->dz};
    double lo[3], d[3];
    double amin = 0.0, amax = 1.0;
    for (int k = 0; k < 3; ++k) {
        lo[k] = -0.5 * n[k] * h[k];
        d[k] = p1[k] - p0[k];
        double hi = lo[k] + n[k] * h[k];
        if (d[k] != 0.0) {
            double a0 = (lo[k] - p0[k]) / d[k], a1 = (hi - p0[k]) / d[k];
            amin = fmax(amin, fmin(a0, a1));
            amax = fmin(amax, fmax(a0, a1));
        } else if (p0[k] < lo[k] || p0[k] >= hi) {
            return 0; /* parallel to this axis and outside the slab */
        }
    }
    if (!(amin < amax)) return 0;

    int m = 0;
    alpha[m++] = amin;
    alpha[m++] = amax;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) continue;
        for (int i = 0; i <= n[k]; ++i) {
            double a = (lo[k] + i * h[k] - p0[k]) / d[k];
            if (a > amin && a < amax) alpha[m++] = a;
        }
    }
    qsort(alpha, (size_t)m, sizeof(double), cmp_double);

    const double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    int cnt = 0;
    for (int t = 0; t + 1 < m; ++t) {
        double a0 = alpha[t], a1 = alpha[t + 1];
        if (!(a1 > a0)) continue; /* coincident crossings: no length */
        double am = 0.5 * (a0 + a1);
        int64_t idx[3];
        int inside = 1;
        for (int k = 0; k < 3; ++k) {
            idx[k] = (int64_t)floor((p0[k] + am * d[k] - lo[k]) / h[k]);
            if (idx[k] < 0 || idx[k] >= n[k]) inside = 0;
        }
        if (!inside) continue;
        vox[cnt] = (idx[2] * g->ny + idx[1]) * g->nx + idx[0];
        len[cnt] = (a1 - a0) * L;
        ++cnt;
    }
    return cnt;
}

/* Index of the voxel's plane along the block axis (z for 3D, y for 2D). */
static int64_t orc_block_coord(const orc_geom *g, int axis, int64_t vox)
{
    if (axis == 2) return vox / ((int64_t)g->nx * g->ny);
    if (axis == 1) return (vox / g->nx) % g->ny;
    return vox % g->nx;
}

static void orc_row_coords(const orc_geom *g, int64_t row, int *a, int *v, int *u)
{
    *u = (int)(row % g->nu);
    *v = (int)((row / g->nu) % g->nv);
    *a = (int)(row / ((int64_t)g->nu * g->nv));
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (called from oracle/bsgd_oracle.py through ctypes). */

int orc_trace_ray(const orc_geom *g, int a, int v, int u, int64_t *vox, double *len, int cap)
{
    if (cap < orc_max_crossings(g)) return -1;
    double p0[3], p1[3];
    double *alpha = (double *)malloc(sizeof(double) * orc_max_crossings(g));
    if (!alpha) return -2;
    orc_ray(g, a, v, u, p0, p1);
    int cnt = orc_trace(g, p0, p1, vox, len, alpha);
    free(alpha);
    return cnt;
}

/*
 * Forward projection of block J = planes [c0, c1) along `axis`, for the listed
 * sinogram rows: out[k] = sum_j A_{rows[k], j} x_j over voxels j in J.
 */
int orc_fp_rows(const orc_geom *g, const double *x, const int64_t *rows, int64_t n_rows,
                int axis, int c0, int c1, double *out)
{
    const int cap = orc_max_crossings(g);
    int err = 0;
#pragma omp parallel
    {
        int64_t *vox = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *alpha = (double *)malloc(sizeof(double) * cap);
        if (!vox || !len || !alpha) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t k = 0; k < n_rows; ++k) {
                int a, v, u;
                double p0[3], p1[3];
                orc_row_coords(g, rows[k], &a, &v, &u);
                orc_ray(g, a, v, u, p0, p1);
                int cnt = orc_trace(g, p0, p1, vox, len, alpha);
                double s = 0.0;
                for (int t = 0; t < cnt; ++t) {
                    int64_t b = orc_block_coord(g, axis, vox[t]);
                    if (b >= c0 && b < c1) s += len[t] * x[vox[t]];
                }
                out[k] = s;
            }
        }
        free(vox); free(len); free(alpha);
    }
    return err ? -2 : 0;
}

/*
 * Back projection of block J: vol[j] += sum_k A_{rows[k], j} r[k] for voxels j
 * in J (vol is the whole volume; voxels outside J are left untouched).
 * Threads scatter into private copies of J that are added up in thread order.
 */
int orc_bp_rows(const orc_geom *g, const double *r, const int64_t *rows, int64_t n_rows,
                int axis, int c0, int c1, double *vol)
{
    if (axis != 1 && axis != 2) return -1;
    const int cap = orc_max_crossings(g);
    const int64_t stride = (axis == 2) ? (int64_t)g->nx * g->ny : (int64_t)g->nx;
    const int64_t base = (int64_t)c0 * stride, span = (int64_t)(c1 - c0) * stride;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *priv = (double *)calloc((size_t)nthr * (size_t)span, sizeof(double));
    if (!priv) return -2;
    int err = 0;
#pragma omp parallel num_threads(nthr)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = priv + (size_t)tid * (size_t)span;
        int64_t *vox = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *alpha = (double *)malloc(sizeof(double) * cap);
        if (!vox || !len || !alpha) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t k = 0; k < n_rows; ++k) {
                int a, v, u;
                double p0[3], p1[3];
                orc_row_coords(g, rows[k], &a, &v, &u);
                orc_ray(g, a, v, u, p0, p1);
                int cnt = orc_trace(g, p0, p1, vox, len, alpha);
                for (int t = 0; t < cnt; ++t) {
                    int64_t b = orc_block_coord(g, axis, vox[t]);
                    if (b >= c0 && b < c1) mine[vox[t] - base] += len[t] * r[k];
                }
            }
        }
        free(vox); free(len); free(alpha);
    }
    if (!err) {
        for (int t = 0; t < nthr; ++t) {
            const double *src = priv + (size_t)t * (size_t)span;
            for (int64_t i = 0; i < span; ++i) vol[base + i] += src[i];
        }
    }
    free(priv);
    return err ? -2 : 0;
}

/*
 * Number of (ray, voxel) pairs for the rows and block J whose length exceeds
 * 1e-4 of the smallest voxel edge. Shorter pieces appear only where a ray
 * passes (up to rounding) through a voxel edge or corner, and have zero length
 * in exact arithmetic.
 */
int64_t orc_count_rows(const orc_geom *g, const int64_t *rows, int64_t n_rows, int axis, int c0, int c1)
{
    const int cap = orc_max_crossings(g);
    const double hmin = fmin(g->dx, fmin(g->dy, g->dz)), eps = 1e-4 * hmin;
    int64_t total = 0;
    int err = 0;
#pragma omp parallel reduction(+ : total)
    {
        int64_t *vox = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *alpha = (double *)malloc(sizeof(double) * cap);
        if (!vox || !len || !alpha) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t k = 0; k < n_rows; ++k) {
                int a, v, u;
                double p0[3], p1[3];
                orc_row_coords(g, rows[k], &a, &v, &u);
                orc_ray(g, a, v, u, p0, p1);
                int cnt = orc_trace(g, p0, p1, vox, len, alpha);
                for (int t = 0; t < cnt; ++t) {
                    int64_t b = orc_block_coord(g, axis, vox[t]);
                    if (b >= c0 && b < c1 && len[t] > eps) total += 1;
                }
            }
        }
        free(vox); free(len); free(alpha);
    }
    return err ? -1 : total;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
