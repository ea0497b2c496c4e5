/*
 * FP64 CPU oracle for the cone-beam operator A of the CT problem, eq. (2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * The paper fixes no discretisation of A (Sec. 3, "Experimental Setup": the
 * projector is taken from a library).  This file writes out the definition
 * that the project uses, one ray at a time, in plain double precision:
 *
 *   geometry   circular cone beam.  View i has angle theta_i = 2*pi*i/n_theta
 *              (uniform over [0, 2*pi), Sec. 3 cases 1-3) unless angles are
 *              given.  Source s = SOD*(cos, sin, 0); detector centre
 *              -(SDD-SOD)*(cos, sin, 0); detector axes e_u = (-sin, cos, 0),
 *              e_v = (0, 0, 1); pixel (iu, iv) centre
 *              c + (iu-(nu-1)/2)*du*e_u + (iv-(nv-1)/2)*dv*e_v; one ray per
 *              pixel through its centre.  Voxel (i, j, k) centre
 *              ((i-(nx-1)/2)*vx, (j-(ny-1)/2)*vy, (k-(nz-1)/2)*vz); volumes
 *              are stored [k][j][i], sinograms [view][iv][iu].
 *   projector  Joseph-type: d = P - s; dominant axis a = argmax |d_a| (ties
 *              go to the lower axis index); for every plane m along a the
 *              crossing point is interpolated bilinearly in the two other
 *              axes with zero outside the volume; the row weight is
 *              v_a * |d| / |d_a|.
 *   adjoint    the exact transpose, formed by scattering every (ray, plane)
 *              tap back into the volume.
 *
 * The per-voxel routine orc_backproject_voxels evaluates single entries of
 * A^T y by brute force over every ray, for checks on volumes too large for a
 * full scatter.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t nx, ny, nz;
    double vx, vy, vz;
    int32_t n_views;
    const double *angles; /* NULL: theta_i = 2*pi*i/n_views */
    double sod, sdd;
    int32_t nu, nv;
    double du, dv;
} orc_geom;

static double view_angle(const orc_geom *g, int v)
{
    return g->angles ? g->angles[v] : 2.0 * M_PI * (double)v / (double)g->n_views;
}

/* Source point s and direction d = P - s of the ray through pixel (iu, iv). */
void orc_ray(const orc_geom *g, int v, int iu, int iv, double s[3], double d[3])
{
    double th = view_angle(g, v);
    double c = cos(th), sn = sin(th);
    double u = ((double)iu - 0.5 * (double)(g->nu - 1)) * g->du;
    double w = ((double)iv - 0.5 * (double)(g->nv - 1)) * g->dv;
    double off = g->sdd - g->sod;
    double P[3];
    s[0] = g->sod * c;
    s[1] = g->sod * sn;
    s[2] = 0.0;
    P[0] = -off * c - u * sn;
    P[1] = -off * sn + u * c;
    P[2] = w;
    d[0] = P[0] - s[0];
    d[1] = P[1] - s[1];
    d[2] = P[2] - s[2];
}

/* Dominant axis of d: the largest |d_a|, the lower index winning ties. */
int orc_dominant_axis(const double d[3])
{
    int a = 0;
    if (fabs(d[1]) > fabs(d[a])) a = 1;
    if (fabs(d[2]) > fabs(d[a])) a = 2;
    return a;
}

/*
 * Taps of one ray on plane m of its dominant axis a: up to four
 * (linear voxel index, bilinear weight) pairs.  Returns how many.
 */
static int plane_taps(const orc_geom *g, const double s[3], const double d[3], int a, int m,
                      int64_t idx[4], double wt[4])
{
    const int N[3] = {g->nx, g->ny, g->nz};
    const double V[3] = {g->vx, g->vy, g->vz};
    int b = (a == 0) ? 1 : 0;
    int c = (a == 2) ? 1 : 2;
    double plane = ((double)m - 0.5 * (double)(N[a] - 1)) * V[a];
    double t = (plane - s[a]) / d[a];
    double qb = (s[b] + t * d[b]) / V[b] + 0.5 * (double)(N[b] - 1);
    double qc = (s[c] + t * d[c]) / V[c] + 0.5 * (double)(N[c] - 1);
    if (!(qb > -1.0 && qb < (double)N[b] && qc > -1.0 && qc < (double)N[c])) return 0;
    double fb0 = floor(qb), fc0 = floor(qc);
    int b0 = (int)fb0, c0 = (int)fc0;
    double fb = qb - fb0, fc = qc - fc0;
    int n = 0;
    for (int db = 0; db < 2; ++db) {
        for (int dc = 0; dc < 2; ++dc) {
            int ib = b0 + db, ic = c0 + dc;
            if (ib < 0 || ib >= N[b] || ic < 0 || ic >= N[c]) continue;
            int ijk[3];
            ijk[a] = m;
            ijk[b] = ib;
            ijk[c] = ic;
            idx[n] = ((int64_t)ijk[2] * N[1] + ijk[1]) * N[0] + ijk[0];
            wt[n] = (db ? fb : 1.0 - fb) * (dc ? fc : 1.0 - fc);
            ++n;
        }
    }
    return n;
}

static double ray_weight(const orc_geom *g, const double d[3], int a)
{
    const double V[3] = {g->vx, g->vy, g->vz};
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    return V[a] * len / fabs(d[a]);
}

/* (A x) for the single ray (v, iu, iv). */
double orc_project_ray(const orc_geom *g, const double *x, int v, int iu, int iv)
{
    double s[3], d[3];
    orc_ray(g, v, iu, iv, s, d);
    int a = orc_dominant_axis(d);
    const int N[3] = {g->nx, g->ny, g->nz};
    double sum = 0.0;
    int64_t idx[4];
    double wt[4];
    for (int m = 0; m < N[a]; ++m) {
        int n = plane_taps(g, s, d, a, m, idx, wt);
        for (int q = 0; q < n; ++q) sum += wt[q] * x[idx[q]];
    }
    return ray_weight(g, d, a) * sum;
}

/* y[s][iv][iu] = (A_S x) for the listed views S (eq. (2.5)'s A_N). */
void orc_project(const orc_geom *g, const double *x, const int32_t *views, int n_sel, double *y)
{
    int64_t per_view = (int64_t)g->nu * g->nv;
    int64_t total = per_view * n_sel;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < total; ++r) {
        int s = (int)(r / per_view);
        int64_t p = r % per_view;
        int iv = (int)(p / g->nu), iu = (int)(p % g->nu);
        y[r] = orc_project_ray(g, x, views[s], iu, iv);
    }
}

/*
 * x = A_S^T y by scattering every tap of every ray.  Each thread scatters a
 * fixed, contiguous block of rays into a private volume; the private volumes
 * are then added in thread order.
 */
int orc_backproject(const orc_geom *g, const double *y, const int32_t *views, int n_sel, double *x)
{
    int64_t nvox = (int64_t)g->nx * g->ny * g->nz;
    int64_t per_view = (int64_t)g->nu * g->nv;
    int64_t total = per_view * n_sel;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *priv = (double *)calloc((size_t)nthreads * (size_t)nvox, sizeof(double));
    if (!priv) return -1;
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0, nt = 1;
#ifdef _OPENMP
        tid = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        double *acc = priv + (size_t)tid * (size_t)nvox;
        int64_t chunk = (total + nt - 1) / nt;
        int64_t r0 = chunk * tid, r1 = r0 + chunk < total ? r0 + chunk : total;
        int64_t idx[4];
        double wt[4];
        for (int64_t r = r0; r < r1; ++r) {
            double yr = y[r];
            if (yr == 0.0) continue;
            int s = (int)(r / per_view);
            int64_t p = r % per_view;
            int iv = (int)(p / g->nu), iu = (int)(p % g->nu);
            double sp[3], d[3];
            orc_ray(g, views[s], iu, iv, sp, d);
            int a = orc_dominant_axis(d);
            const int N[3] = {g->nx, g->ny, g->nz};
            double wy = ray_weight(g, d, a) * yr;
            for (int m = 0; m < N[a]; ++m) {
                int n = plane_taps(g, sp, d, a, m, idx, wt);
                for (int q = 0; q < n; ++q) acc[idx[q]] += wt[q] * wy;
            }
        }
    }
    memset(x, 0, (size_t)nvox * sizeof(double));
    for (int t = 0; t < nthreads; ++t) {
        const double *acc = priv + (size_t)t * (size_t)nvox;
        for (int64_t q = 0; q < nvox; ++q) x[q] += acc[q];
    }
    free(priv);
    return 0;
}

/*
 * Single entries (A_S^T y)_j for the listed linear voxel indices, by brute
 * force: every ray of every listed view is visited and, on the plane of its
 * dominant axis that contains voxel j, the tap weight of voxel j is taken.
 */
void orc_backproject_voxels(const orc_geom *g, const double *y, const int32_t *views, int n_sel,
                            const int64_t *vox, int n_vox, double *out)
{
    const int N[3] = {g->nx, g->ny, g->nz};
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < n_vox; ++q) {
        int64_t j = vox[q];
        int ijk[3];
        ijk[0] = (int)(j % N[0]);
        ijk[1] = (int)((j / N[0]) % N[1]);
        ijk[2] = (int)(j / ((int64_t)N[0] * N[1]));
        double sum = 0.0;
        int64_t idx[4];
        double wt[4];
        for (int s = 0; s < n_sel; ++s) {
            for (int iv = 0; iv < g->nv; ++iv) {
                for (int iu = 0; iu < g->nu; ++iu) {
                    double yr = y[((int64_t)s * g->nv + iv) * g->nu + iu];
                    if (yr == 0.0) continue;
                    double sp[3], d[3];
                    orc_ray(g, views[s], iu, iv, sp, d);
                    int a = orc_dominant_axis(d);
                    int n = plane_taps(g, sp, d, a, ijk[a], idx, wt);
                    for (int t = 0; t < n; ++t)
                        if (idx[t] == j) sum += ray_weight(g, d, a) * wt[t] * yr;
                }
            }
        }
        out[q] = sum;
    }
}

/* Number of threads the oracle's parallel loops use. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
