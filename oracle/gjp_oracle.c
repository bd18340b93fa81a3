/*
 * gjp_oracle.c -- plain FP64 CPU reference of the branchless generalized
 * Joseph projector (GJP), J. Graetz, "High performance volume ray casting:
 * A branchless generalized Joseph projector".
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header
 * or constant with the CUDA library, and the library never calls it.
 *
 * Forward projection follows Algorithm 1 in the paper's order and notation,
 * evaluated in double precision, one ray at a time:
 *
 *   s, d       source and pixel centre in voxel-index units      (Eq. 1-2)
 *   r = d - s                                                     (Eq. 2)
 *   m = argmax_k |r_k|                                            (Eq. 3)
 *   rt = r / r_m                                                  (Eq. 4)
 *   o = -s_m                                                      (Eq. 5)
 *   p(i) = s + (o + i) rt, i = 0 .. n_m - 1                       (Eq. 6)
 *   four taps from floor/ceil combinations                        (Eq. 7-8)
 *   w_fl,k = w(p_k - floor p_k), w_cl,k = 1 - w_fl,k,
 *   w_fl,m = w_cl,m = 1                                           (Eq. 10-11)
 *   tap weights w_fl/cl,1 * w_fl/cl,2 * w_fl/cl,3                  (Eq. 12)
 *   w_lin(d) = 1 - d  /  w_spl(d) = 1 - 3d^2 + 2d^3               (Eq. 13-14)
 *   a += volume[tap] * |rt| * weight                              (Algorithm 1)
 *
 * Readings where the paper is silent or loose (each listed in the design
 * notes of the repository):
 *   C1  the driving-axis component of p(i) is set to the integer i exactly,
 *       which Algorithm 1 asserts holds by construction;
 *   C2  argmax ties go to the lowest axis index; callers may force m;
 *   C3  "p is in volume" is read per tap: a tap contributes iff each of its
 *       indices lies in [0, n_k - 1] (zero border);
 *   C4  the step weight is |h (.) rt| (world length per plane step) for
 *       voxel size h, which is |rt| for unit voxels;
 *   C5  the line is integrated over the whole volume (source and detector
 *       lie outside it);
 *   C6  voxel centres sit on integer indices, world = origin + index * h;
 *       pixel centre = det_origin + iu * det_u + iv * det_v.
 *
 * The adjoint is the literal transpose: the same loop, scattering
 * y * |h (.) rt| * weight into the taps (the system-matrix view of the
 * reconstruction section, g = A f).
 *
 * The analytic ellipsoid projector gives closed-form line integrals of a sum
 * of ellipsoids, averaged over a regular sub-pixel grid of rays per detector
 * pixel, as used for the reference projections of the projection-quality
 * experiment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_F64 = 0, ORACLE_F32 = 1 };

typedef struct {
    const void *vol;
    int dtype;
    int64_t n[3];
    double h[3];
    double origin[3];
    int wfun; /* 0 = w_lin (Eq. 13), 1 = w_spl (Eq. 14) */
    double fov; /* > 0: sample only inside the cylinder of this radius (see below) */
} oracle_volume;

/*
 * Field-of-view cylinder of the paper's speed benchmark: the sampling points
 * of each ray are restricted to its intersection with a cylinder around the
 * rotation axis (here: the line through the volume centre parallel to z, of
 * world radius fov) instead of the bounding box.  A plane's sample p (index
 * units) is kept iff its world distance from that axis is at most fov.
 */
static int outside_fov(const oracle_volume *V, const double p[3])
{
    if (!(V->fov > 0.0)) return 0;
    const double dx = V->h[0] * (p[0] - 0.5 * (double)(V->n[0] - 1));
    const double dy = V->h[1] * (p[1] - 0.5 * (double)(V->n[1] - 1));
    return dx * dx + dy * dy > V->fov * V->fov;
}

static double vol_at(const oracle_volume *V, int64_t i, int64_t j, int64_t k)
{
    const int64_t idx = (i * V->n[1] + j) * V->n[2] + k;
    if (V->dtype == ORACLE_F64) return ((const double *)V->vol)[idx];
    return (double)((const float *)V->vol)[idx];
}

/* Eq. 13 / Eq. 14 */
static double weight_fn(int wfun, double d)
{
    if (wfun == 1) return 1.0 - 3.0 * d * d + 2.0 * d * d * d;
    return 1.0 - d;
}

/* Eq. 3 with ties to the lowest index (reading C2) */
static int driving_axis(const double r[3])
{
    int m = 0;
    for (int k = 1; k < 3; ++k)
        if (fabs(r[k]) > fabs(r[m])) m = k;
    return m;
}

/* Source and pixel centre of one ray in voxel-index units (Eq. 1-2, C6). */
static void ray_endpoints(const oracle_volume *V, const double *src, const double *det_origin,
                          const double *det_u, const double *det_v, int view, double iu, double iv,
                          double s[3], double d[3])
{
    for (int k = 0; k < 3; ++k) {
        const double pix = det_origin[3 * view + k] + iu * det_u[3 * view + k] + iv * det_v[3 * view + k];
        s[k] = (src[3 * view + k] - V->origin[k]) / V->h[k];
        d[k] = (pix - V->origin[k]) / V->h[k];
    }
}

/*
 * One ray of Algorithm 1.  If y_scatter is NULL the ray's line integral is
 * returned; otherwise y is scattered into out_vol (adjoint) and 0 returned.
 * force_m < 0 selects m by Eq. 3, otherwise m = force_m.
 */
static double gjp_ray(const oracle_volume *V, const double s[3], const double d[3], int force_m,
                      const double *y_scatter, double *out_vol)
{
    double r[3], rt[3];
    for (int k = 0; k < 3; ++k) r[k] = d[k] - s[k];                    /* Eq. 2 */
    const int m = force_m >= 0 ? force_m : driving_axis(r);            /* Eq. 3 */
    if (r[m] == 0.0) return 0.0;
    for (int k = 0; k < 3; ++k) rt[k] = r[k] / r[m];                   /* Eq. 4 */
    const double o = -s[m];                                            /* Eq. 5 */
    const int64_t imax = V->n[m];                                      /* number of planes */
    double hr2 = 0.0;                                                  /* |h (.) rt|, C4 */
    for (int k = 0; k < 3; ++k) hr2 += (V->h[k] * rt[k]) * (V->h[k] * rt[k]);
    const double step = sqrt(hr2);

    double a = 0.0;
    for (int64_t i = 0; i < imax; ++i) {
        double p[3], pfl[3], pcl[3], wfl[3], wcl[3];
        for (int k = 0; k < 3; ++k) p[k] = s[k] + (o + (double)i) * rt[k]; /* Eq. 6 */
        p[m] = (double)i;                                               /* C1 */
        if (outside_fov(V, p)) continue;
        for (int k = 0; k < 3; ++k) {
            pfl[k] = floor(p[k]);                                       /* Eq. 7 */
            pcl[k] = ceil(p[k]);
            wfl[k] = weight_fn(V->wfun, p[k] - pfl[k]);                 /* Eq. 10-11 */
            wcl[k] = 1.0 - wfl[k];
        }
        wfl[m] = wcl[m] = 1.0;                                          /* Eq. 11, k = m */
        /* the four neighbours of Eq. 7 and their weights (Eq. 12) */
        const double *sel[4][3] = {
            {&pfl[0], &pfl[1], &pfl[2]},
            {&pfl[0], &pcl[1], &pcl[2]},
            {&pcl[0], &pfl[1], &pcl[2]},
            {&pcl[0], &pcl[1], &pfl[2]},
        };
        const double w4[4] = {
            wfl[0] * wfl[1] * wfl[2],
            wfl[0] * wcl[1] * wcl[2],
            wcl[0] * wfl[1] * wcl[2],
            wcl[0] * wcl[1] * wfl[2],
        };
        for (int t = 0; t < 4; ++t) {
            int64_t idx[3];
            int inside = 1;
            for (int k = 0; k < 3; ++k) {
                const double v = *sel[t][k];
                if (v < 0.0 || v > (double)(V->n[k] - 1)) inside = 0;   /* C3 */
                idx[k] = inside ? (int64_t)v : 0;
            }
            if (!inside) continue;
            if (y_scatter) {
                out_vol[(idx[0] * V->n[1] + idx[1]) * V->n[2] + idx[2]] += (*y_scatter) * step * w4[t];
            } else {
                a += vol_at(V, idx[0], idx[1], idx[2]) * step * w4[t];
            }
        }
    }
    return a;
}

static int check_volume(const oracle_volume *V)
{
    if (!V->vol && V->dtype >= 0) return 1;
    for (int k = 0; k < 3; ++k)
        if (V->n[k] <= 0 || !(V->h[k] > 0.0)) return 1;
    if (V->dtype != ORACLE_F64 && V->dtype != ORACLE_F32) return 1;
    if (V->wfun != 0 && V->wfun != 1) return 1;
    return 0;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/*
 * Forward projection of every pixel of every view.
 * proj: [n_views][nv][nu] doubles, iu fastest.
 */
int gjp_oracle_forward(const void *vol, int vol_dtype, int64_t nx, int64_t ny, int64_t nz,
                       const double h[3], const double origin[3], int n_views, int nu, int nv,
                       const double *src, const double *det_origin, const double *det_u,
                       const double *det_v, int wfun, double fov, int nthreads, double *proj)
{
    oracle_volume V = {vol, vol_dtype, {nx, ny, nz}, {h[0], h[1], h[2]},
                       {origin[0], origin[1], origin[2]}, wfun, fov};
    if (check_volume(&V) || n_views < 0 || nu <= 0 || nv <= 0 || !proj) return 1;
    set_threads(nthreads);
    const int64_t n_rays = (int64_t)n_views * nv * nu;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t ray = 0; ray < n_rays; ++ray) {
        const int view = (int)(ray / ((int64_t)nv * nu));
        const int iv = (int)((ray / nu) % nv);
        const int iu = (int)(ray % nu);
        double s[3], d[3];
        ray_endpoints(&V, src, det_origin, det_u, det_v, view, iu, iv, s, d);
        proj[ray] = gjp_ray(&V, s, d, -1, NULL, NULL);
    }
    return 0;
}

/*
 * Forward projection of selected rays (view[j], iu[j], iv[j]); axis may be
 * NULL, or give per ray -1 (Eq. 3) or a forced driving axis 0..2.
 */
int gjp_oracle_rays(const void *vol, int vol_dtype, int64_t nx, int64_t ny, int64_t nz,
                    const double h[3], const double origin[3], const double *src,
                    const double *det_origin, const double *det_u, const double *det_v,
                    int64_t n_rays, const int32_t *view, const int32_t *iu, const int32_t *iv,
                    const int32_t *axis, int wfun, double fov, int nthreads, double *out)
{
    oracle_volume V = {vol, vol_dtype, {nx, ny, nz}, {h[0], h[1], h[2]},
                       {origin[0], origin[1], origin[2]}, wfun, fov};
    if (check_volume(&V) || n_rays < 0 || !out) return 1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < n_rays; ++j) {
        double s[3], d[3];
        ray_endpoints(&V, src, det_origin, det_u, det_v, view[j], iu[j], iv[j], s, d);
        const int fm = axis ? axis[j] : -1;
        out[j] = (fm > 2) ? NAN : gjp_ray(&V, s, d, fm, NULL, NULL);
    }
    return 0;
}

/*
 * Per-ray setup quantities, for pins and for the tie rule: driving axis m
 * (Eq. 3), rt (Eq. 4) and the relative argmax margin
 * (|r|_(1) - |r|_(2)) / |r|.
 */
int gjp_oracle_ray_info(int64_t nx, int64_t ny, int64_t nz, const double h[3], const double origin[3],
                        const double *src, const double *det_origin, const double *det_u,
                        const double *det_v, int64_t n_rays, const int32_t *view,
                        const int32_t *iu, const int32_t *iv, int32_t *m_out, double *rt_out,
                        double *margin_out)
{
    oracle_volume V = {NULL, -1, {nx, ny, nz}, {h[0], h[1], h[2]},
                       {origin[0], origin[1], origin[2]}, 0, 0.0};
    for (int64_t j = 0; j < n_rays; ++j) {
        double s[3], d[3], r[3], a[3];
        ray_endpoints(&V, src, det_origin, det_u, det_v, view[j], iu[j], iv[j], s, d);
        for (int k = 0; k < 3; ++k) {
            r[k] = d[k] - s[k];
            a[k] = fabs(r[k]);
        }
        const int m = driving_axis(r);
        m_out[j] = m;
        for (int k = 0; k < 3; ++k) rt_out[3 * j + k] = r[k] / r[m];
        double second = 0.0;
        for (int k = 0; k < 3; ++k)
            if (k != m && a[k] > second) second = a[k];
        margin_out[j] = (a[m] - second) / sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    }
    return 0;
}

/*
 * Adjoint (transpose) of gjp_oracle_forward: vol_out += A^T proj.
 * vol_out: [nx][ny][nz] doubles; the caller zeroes it for a plain A^T y.
 * With nthreads > 1 each thread scatters into a private copy that is summed
 * afterwards; the thread count is reduced until the copies fit in max_bytes.
 */
int gjp_oracle_adjoint(const double *proj, int64_t nx, int64_t ny, int64_t nz, const double h[3],
                       const double origin[3], int n_views, int nu, int nv, const double *src,
                       const double *det_origin, const double *det_u, const double *det_v,
                       int wfun, double fov, int nthreads, double max_bytes, double *vol_out)
{
    oracle_volume V = {NULL, -1, {nx, ny, nz}, {h[0], h[1], h[2]},
                       {origin[0], origin[1], origin[2]}, wfun, fov};
    for (int k = 0; k < 3; ++k)
        if (V.n[k] <= 0 || !(V.h[k] > 0.0)) return 1;
    if (!proj || !vol_out || n_views < 0 || nu <= 0 || nv <= 0) return 1;
    const int64_t nvox = nx * ny * nz;
    const int64_t n_rays = (int64_t)n_views * nv * nu;
    int T = 1;
#ifdef _OPENMP
    T = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    if (T > 1 && (double)T * (double)nvox * 8.0 > max_bytes) {
        T = (int)(max_bytes / ((double)nvox * 8.0));
        if (T < 1) T = 1;
    }
    if (T <= 1) {
        for (int64_t ray = 0; ray < n_rays; ++ray) {
            const int view = (int)(ray / ((int64_t)nv * nu));
            const int iv = (int)((ray / nu) % nv);
            const int iu = (int)(ray % nu);
            double s[3], d[3];
            ray_endpoints(&V, src, det_origin, det_u, det_v, view, iu, iv, s, d);
            gjp_ray(&V, s, d, -1, &proj[ray], vol_out);
        }
        return 0;
    }
    double *priv = (double *)calloc((size_t)T * (size_t)nvox, sizeof(double));
    if (!priv) return 2;
    set_threads(T);
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = priv + (size_t)tid * (size_t)nvox;
#pragma omp for schedule(dynamic, 64)
        for (int64_t ray = 0; ray < n_rays; ++ray) {
            const int view = (int)(ray / ((int64_t)nv * nu));
            const int iv = (int)((ray / nu) % nv);
            const int iu = (int)(ray % nu);
            double s[3], d[3];
            ray_endpoints(&V, src, det_origin, det_u, det_v, view, iu, iv, s, d);
            gjp_ray(&V, s, d, -1, &proj[ray], mine);
        }
#pragma omp for schedule(static)
        for (int64_t v = 0; v < nvox; ++v) {
            double acc = 0.0;
            for (int t = 0; t < T; ++t) acc += priv[(size_t)t * (size_t)nvox + v];
            vol_out[v] += acc;
        }
    }
    free(priv);
    return 0;
}

/*
 * Closed-form line integrals of a sum of ellipsoids (the analytic reference
 * projections of the projection-quality experiment).  Each pixel value is
 * the mean over sub x sub rays from the source to cell-centred points
 * (iu + (a + 1/2)/sub - 1/2, iv + (b + 1/2)/sub - 1/2) of the pixel.
 * Ellipsoid record (16 doubles): rho, c[3], semi-axes[3], R[9] row-major
 * with the principal axes as columns; inside iff |diag(1/a) R^T (x-c)| <= 1.
 * The chord of the full line through each ellipsoid is its world length.
 */
int gjp_oracle_ellipsoid_project(int n_ell, const double *ell, int n_views, int nu, int nv,
                                 const double *src, const double *det_origin, const double *det_u,
                                 const double *det_v, int sub, int nthreads, double *proj)
{
    if (n_ell < 0 || n_views < 0 || nu <= 0 || nv <= 0 || sub <= 0 || !proj) return 1;
    set_threads(nthreads);
    const int64_t n_rays = (int64_t)n_views * nv * nu;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t ray = 0; ray < n_rays; ++ray) {
        const int view = (int)(ray / ((int64_t)nv * nu));
        const int iv = (int)((ray / nu) % nv);
        const int iu = (int)(ray % nu);
        const double *S = src + 3 * view;
        double total = 0.0;
        for (int a = 0; a < sub; ++a) {
            for (int b = 0; b < sub; ++b) {
                const double fu = iu + (a + 0.5) / sub - 0.5;
                const double fv = iv + (b + 0.5) / sub - 0.5;
                double dir[3];
                for (int k = 0; k < 3; ++k)
                    dir[k] = det_origin[3 * view + k] + fu * det_u[3 * view + k] +
                             fv * det_v[3 * view + k] - S[k];
                const double len = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
                for (int e = 0; e < n_ell; ++e) {
                    const double *E = ell + 16 * e;
                    const double *c = E + 1, *ax = E + 4, *R = E + 7;
                    double u0[3], q[3];
                    for (int k = 0; k < 3; ++k) {
                        u0[k] = (R[0 * 3 + k] * (S[0] - c[0]) + R[1 * 3 + k] * (S[1] - c[1]) +
                                 R[2 * 3 + k] * (S[2] - c[2])) / ax[k];
                        q[k] = (R[0 * 3 + k] * dir[0] + R[1 * 3 + k] * dir[1] + R[2 * 3 + k] * dir[2]) / ax[k];
                    }
                    /* |u0 + t q|^2 = 1 */
                    const double A = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
                    const double B = u0[0] * q[0] + u0[1] * q[1] + u0[2] * q[2];
                    const double C = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2] - 1.0;
                    const double disc = B * B - A * C;
                    if (disc <= 0.0) continue;
                    const double dt = 2.0 * sqrt(disc) / A; /* t2 - t1 */
                    total += E[0] * dt * len;
                }
            }
        }
        proj[ray] = total / ((double)sub * sub);
    }
    return 0;
}
