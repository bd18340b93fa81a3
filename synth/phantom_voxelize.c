/*
 * Supersampled rasterisation of a sum of ellipsoids onto a voxel grid
 * (input generation for tests and benchmarks; no projector arithmetic).
 *
 * Each voxel value is the mean, over s*s*s regularly placed sub-samples
 * at cell-centred offsets (a + 1/2)/s - 1/2 (in voxel units) around the
 * voxel centre, of the phantom function sum_e rho_e * [x inside e].
 * Points exactly on an ellipsoid surface count as inside.  This is the
 * rasterisation with supersampling described with the 3-D Shepp-Logan
 * phantom in the paper's projection-quality section.
 *
 * Ellipsoid record (16 doubles): rho, c[3], a[3], R[9] (row-major 3x3 whose
 * columns are the principal axes in world coordinates).  A point x is
 * inside iff |diag(1/a) R^T (x - c)| <= 1.
 *
 * For speed the z direction is handled per sub-sample column: for a fixed
 * (x, y) the inside set along z is one closed interval (a quadratic
 * inequality), whose sub-sample index range is accumulated with a
 * difference array.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int phantom_voxelize(int n_ell, const double *ell, int64_t nx, int64_t ny, int64_t nz,
                     const double h[3], const double origin[3], int s, float *out,
                     int nthreads)
{
    if (n_ell < 0 || nx <= 0 || ny <= 0 || nz <= 0 || s <= 0 || !out) return 1;
    const int64_t nzs = nz * s;
    const double inv_s3 = 1.0 / ((double)s * s * s);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif

#pragma omp parallel
    {
        double *diff = (double *)malloc(sizeof(double) * (size_t)(nzs + 1));
        double *col = (double *)malloc(sizeof(double) * (size_t)nz);
#pragma omp for schedule(dynamic, 1)
        for (int64_t ij = 0; ij < nx * ny; ++ij) {
            const int64_t i = ij / ny, j = ij % ny;
            memset(col, 0, sizeof(double) * (size_t)nz);
            for (int a = 0; a < s; ++a) {
                const double X = origin[0] + (i + (a + 0.5) / s - 0.5) * h[0];
                for (int b = 0; b < s; ++b) {
                    const double Y = origin[1] + (j + (b + 0.5) / s - 0.5) * h[1];
                    memset(diff, 0, sizeof(double) * (size_t)(nzs + 1));
                    int any = 0;
                    for (int e = 0; e < n_ell; ++e) {
                        const double *E = ell + 16 * e;
                        const double rho = E[0];
                        const double *c = E + 1, *ax = E + 4, *R = E + 7;
                        /* u0 = diag(1/a) R^T (X - cx, Y - cy, -cz), q = diag(1/a) R^T e_z */
                        const double dx = X - c[0], dy = Y - c[1], dz = -c[2];
                        double u0[3], q[3];
                        for (int k = 0; k < 3; ++k) {
                            u0[k] = (R[0 * 3 + k] * dx + R[1 * 3 + k] * dy + R[2 * 3 + k] * dz) / ax[k];
                            q[k] = R[2 * 3 + k] / ax[k];
                        }
                        const double A = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
                        const double B = u0[0] * q[0] + u0[1] * q[1] + u0[2] * q[2];
                        const double C = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2] - 1.0;
                        const double disc = B * B - A * C;
                        if (disc < 0.0) continue;
                        const double sq = sqrt(disc);
                        const double z0 = (-B - sq) / A, z1 = (-B + sq) / A; /* world z */
                        /* sub-sample g sits at z_g = origin_z + ((g + 1/2)/s - 1/2) h_z */
                        double g0 = ceil(((z0 - origin[2]) / h[2] + 0.5) * s - 0.5);
                        double g1 = floor(((z1 - origin[2]) / h[2] + 0.5) * s - 0.5);
                        if (g0 < 0) g0 = 0;
                        if (g1 > (double)(nzs - 1)) g1 = (double)(nzs - 1);
                        if (g1 < g0) continue;
                        diff[(int64_t)g0] += rho;
                        diff[(int64_t)g1 + 1] -= rho;
                        any = 1;
                    }
                    if (!any) continue;
                    double run = 0.0;
                    for (int64_t g = 0; g < nzs; ++g) {
                        run += diff[g];
                        col[g / s] += run;
                    }
                }
            }
            float *dst = out + (i * ny + j) * nz;
            for (int64_t k = 0; k < nz; ++k) {
                /* the running sum of +rho/-rho steps can leave ~1e-16 where the
                   exact value is 0; snap those so empty space is exactly zero */
                const double v = col[k] * inv_s3;
                dst[k] = (float)(fabs(v) < 1e-12 ? 0.0 : v);
            }
        }
        free(diff);
        free(col);
    }
    return 0;
}
