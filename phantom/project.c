/*
 * Seeded-input generator: closed-form line integrals of ellipsoid phantoms
 * on a circular cone-beam orbit.  This is test-data generation only; it
 * holds none of the reconstruction method's arithmetic (no filtering, no
 * bounds, no decimation, no backprojection) and is the one input source
 * shared by the oracle and the CUDA path.
 *
 * Geometry (the reading used throughout the project):
 *   angle          beta_k = 2*pi*k/P, k = 0..P-1 (full orbit, Sec. 2.2)
 *   source         S = -R (cos beta, sin beta, 0)
 *   virtual detector through the isocentre, pitch 1 voxel:
 *                  point T(a,b) = a*(-sin beta, cos beta, 0) + b*(0,0,1)
 *                  a = u - (Nu-1)/2,  b = v - (Nv-1)/2
 *   ray            S + lambda (T - S)
 * which puts the projection of a point (x,y) at the column of Eq. 1.
 *
 * Ellipsoid e: centre c, rotation Q (columns = body axes in the world
 * frame), semi-axes (A,B,C), density rho.  Mapped to the unit sphere,
 * p' = diag(1/A,1/B,1/C) Q^T (p - c).  With s' and d' the mapped source and
 * ray direction, the chord parameter length is
 *   2 sqrt((s'.d')^2 - |d'|^2 (|s'|^2 - 1)) / |d'|^2
 * and the physical chord is that times |T - S| = sqrt(R^2 + a^2 + b^2).
 *
 * Parameter block per ellipsoid (16 doubles):
 *   cx cy cz  A B C  q00 q01 q02 q10 q11 q12 q20 q21 q22  rho
 * (q row-major, column j = body axis j).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

#define NPAR 16

static void mapvec(const double *e, const double *v, double *out) {
    const double *q = e + 6; /* out = diag(1/A,1/B,1/C) Q^T v */
    double r0 = q[0] * v[0] + q[3] * v[1] + q[6] * v[2];
    double r1 = q[1] * v[0] + q[4] * v[1] + q[7] * v[2];
    double r2 = q[2] * v[0] + q[5] * v[1] + q[8] * v[2];
    out[0] = r0 / e[3];
    out[1] = r1 / e[4];
    out[2] = r2 / e[5];
}

static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* One detector row (angle k, row v) into acc[0..Nu-1] (double). */
static void project_row(int n_ell, const double *ell, double R, int Nu, int Nv,
                        int P, int k, int v, double *acc) {
    const double uc = 0.5 * (double)(Nu - 1), vc = 0.5 * (double)(Nv - 1);
    double beta = 2.0 * M_PI * (double)k / (double)P;
    double cb = cos(beta), sb = sin(beta);
    double S[3] = {-R * cb, -R * sb, 0.0};
    double n[3] = {R * cb, R * sb, 0.0}; /* T(0,0) - S */
    double eu[3] = {-sb, cb, 0.0};
    double ez[3] = {0.0, 0.0, 1.0};
    double b = (double)v - vc;
    for (int u = 0; u < Nu; ++u) acc[u] = 0.0;
    for (int e = 0; e < n_ell; ++e) {
        const double *E = ell + (size_t)e * NPAR;
        double sc[3] = {S[0] - E[0], S[1] - E[1], S[2] - E[2]};
        double sp[3], np_[3], eup[3], ezp[3];
        mapvec(E, sc, sp);
        mapvec(E, n, np_);
        mapvec(E, eu, eup);
        mapvec(E, ez, ezp);
        double ss1 = dot3(sp, sp) - 1.0;
        double rho = E[15];
        double d0[3] = {np_[0] + b * ezp[0], np_[1] + b * ezp[1], np_[2] + b * ezp[2]};
        /* disc(a) = q2 a^2 + 2 q1 a + q0: find the a-interval where it is > 0
         * to skip columns the ellipsoid cannot touch (values are still
         * evaluated per ray below). */
        double s0 = dot3(sp, d0), s1 = dot3(sp, eup);
        double q2 = s1 * s1 - ss1 * dot3(eup, eup);
        double q1 = s0 * s1 - ss1 * dot3(d0, eup);
        double q0 = s0 * s0 - ss1 * dot3(d0, d0);
        int ulo = 0, uhi = Nu - 1;
        if (q2 < 0.0) {
            double dq = q1 * q1 - q2 * q0;
            if (dq <= 0.0) continue;
            double r = sqrt(dq);
            double a1 = (-q1 + r) / q2, a2 = (-q1 - r) / q2;
            double alo = a1 < a2 ? a1 : a2, ahi = a1 < a2 ? a2 : a1;
            double flo = floor(alo + uc) - 1.0, fhi = ceil(ahi + uc) + 1.0;
            if (fhi < 0.0 || flo > (double)(Nu - 1)) continue;
            ulo = flo < 0.0 ? 0 : (int)flo;
            uhi = fhi > (double)(Nu - 1) ? Nu - 1 : (int)fhi;
        }
        for (int u = ulo; u <= uhi; ++u) {
            double a = (double)u - uc;
            double dp[3] = {d0[0] + a * eup[0], d0[1] + a * eup[1], d0[2] + a * eup[2]};
            double sd = dot3(sp, dp), dd = dot3(dp, dp);
            double disc = sd * sd - dd * ss1;
            if (disc > 0.0) {
                double dlen = sqrt(R * R + a * a + b * b);
                acc[u] += rho * dlen * 2.0 * sqrt(disc) / dd;
            }
        }
    }
}

static int bad_args(int n_ell, int Nu, int Nv, int P, int k0, int k1) {
    return n_ell < 0 || Nu <= 0 || Nv <= 0 || P <= 0 || k0 < 0 || k1 > P || k0 > k1;
}

/* Projections for angles k0..k1-1 into out[(k-k0)][v][u], double. */
int phantom_project_f64(int n_ell, const double *ell, double R, int Nu, int Nv,
                        int P, int k0, int k1, double *out) {
    if (bad_args(n_ell, Nu, Nv, P, k0, k1)) return -1;
    long rows = (long)(k1 - k0) * Nv;
#pragma omp parallel for schedule(dynamic, 4)
    for (long r = 0; r < rows; ++r) {
        int kk = (int)(r / Nv), v = (int)(r % Nv);
        project_row(n_ell, ell, R, Nu, Nv, P, k0 + kk, v, out + (size_t)r * Nu);
    }
    return 0;
}

/* Detector rows v0..v1-1 only, for angles k0..k1-1, rounded to float32:
 * out[(k-k0)][v-v0][u] (the rows a bounded sample of slices reads). */
int phantom_project_band_f32(int n_ell, const double *ell, double R, int Nu, int Nv, int P, int k0, int k1,
                             int v0, int v1, float *out) {
    if (bad_args(n_ell, Nu, Nv, P, k0, k1) || v0 < 0 || v1 > Nv || v0 > v1) return -1;
    const int nb = v1 - v0;
    long rows = (long)(k1 - k0) * nb;
    int fail = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)Nu);
        if (!acc) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (long r = 0; r < rows; ++r) {
            if (!acc) continue;
            int kk = (int)(r / nb), v = v0 + (int)(r % nb);
            project_row(n_ell, ell, R, Nu, Nv, P, k0 + kk, v, acc);
            float *row = out + (size_t)r * Nu;
            for (int u = 0; u < Nu; ++u) row[u] = (float)acc[u];
        }
        free(acc);
    }
    return fail ? -2 : 0;
}

/* Same, rounded to float32 (the pipeline's input precision). */
int phantom_project_f32(int n_ell, const double *ell, double R, int Nu, int Nv,
                        int P, int k0, int k1, float *out) {
    if (bad_args(n_ell, Nu, Nv, P, k0, k1)) return -1;
    long rows = (long)(k1 - k0) * Nv;
    int fail = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)Nu);
        if (!acc) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (long r = 0; r < rows; ++r) {
            if (!acc) continue;
            int kk = (int)(r / Nv), v = (int)(r % Nv);
            project_row(n_ell, ell, R, Nu, Nv, P, k0 + kk, v, acc);
            float *row = out + (size_t)r * Nu;
            for (int u = 0; u < Nu; ++u) row[u] = (float)acc[u];
        }
        free(acc);
    }
    return fail ? -2 : 0;
}
