/*
 * FP64 CPU oracle for FDK and FDK-OD (Andriiashen & Kozhevnikov, "Fast
 * optimal decomposed modification of FDK").
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines what the CUDA library must
 * compute; it shares no code, header or table with the CUDA path and is
 * used only by the test-suite, the smoke check and the CPU baseline leg of
 * the benchmark.  It is deliberately plain and slow: every step is written
 * in the paper's order, in FP64, with no blocking or fusion.  It must be
 * compiled with -ffp-contract=off so that the integer crop bounds are
 * reproducible bit for bit.
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *  - voxel centres x_i = i - (N-1)/2 (same for y, z), voxel size 1;
 *  - virtual flat detector through the isocentre, pitch 1,
 *    a = u - (Nu-1)/2, b = v - (Nv-1)/2;
 *  - R in Eq. 1 is the source-to-isocentre distance, beta_k = 2 pi k / P
 *    over a full orbit (Sec. 2.2 lets beta run over 360 degrees);
 *  - filter: textbook FDK cosine weight R / sqrt(R^2 + a^2 + b^2) and the
 *    discrete Ram-Lak kernel (unit sample spacing), linear convolution with
 *    zero padding (the paper calls this the initial convolution, Sec. 1);
 *  - backprojection weight U^-2 with U = (R + x cos b + y sin b) / R and
 *    scale pi / P (half the angular step of a full orbit);
 *  - square decomposition: voxel i belongs to square floor(i 2^s / N)
 *    (Sec. 2.2, squares of side N / 2^s); the vertices are the centres of
 *    the square's corner voxels;
 *  - shift centre: the projection of the square centre,
 *    phi_k = a(x_c, y_c, beta_k) + (Nu-1)/2;
 *  - angular decimation: triangle low-pass with taps (D - |i|) / D^2,
 *    |i| < D, circular over the full orbit, then keep every D-th angle
 *    (Sec. 2.1: low-pass filter, then downsample).  Sec. 2.1 leaves the
 *    filter open (its quality "can be adjusted"), so any symmetric taps
 *    h[|i|], |i| < H D, may be passed instead (h = NULL: the triangle);
 *  - the second shift back to original positions is folded into the
 *    backprojection's column coordinate (Sec. 2.2 says FDK-OD performs a
 *    single interpolation);
 *  - samples outside the detector are zero; bilinear interpolation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2
#define ORACLE_ECROP -3 /* a D=1 read fell outside its square's crop window */

/* ---------------------------------------------------------------- basics */

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Projection angle of view k on a full circular orbit. */
static double beta_of(int k, int P) { return 2.0 * M_PI * (double)k / (double)P; }

/* Eq. 1: detector column (isocentre units) of the point (x, y) at the angle
 * with cosine cb and sine sb.  Written left to right exactly as printed. */
static double eq1_a(double R, double x, double y, double cb, double sb) {
    double num = y * cb - x * sb;
    double den = R + x * cb + y * sb;
    return R * num / den;
}

/* Magnification factor U = (R + x cos b + y sin b) / R of the FDK weight. */
static double fdk_U(double R, double x, double y, double cb, double sb) {
    return (R + x * cb + y * sb) / R;
}

/* Voxel-centre coordinate of index i in a grid of n. */
static double centre(int i, int n) { return (double)i - 0.5 * (double)(n - 1); }

/* First and last voxel index of square q along one axis (voxel i belongs to
 * square floor(i 2^s / N)). */
static void square_range(int q, int s, int N, int *i0, int *i1) {
    long m = 1L << s;
    *i0 = (int)(((long)q * N + m - 1) / m);
    *i1 = (int)((((long)q + 1) * N + m - 1) / m) - 1;
}

/* ---------------------------------------------------------------- filter */

/* Discrete Ram-Lak kernel with unit sample spacing. */
static double ramlak(long n) {
    if (n == 0) return 0.25;
    if (n % 2 == 0) return 0.0;
    double dn = (double)n;
    return -1.0 / (M_PI * M_PI * dn * dn);
}

/* Filter the detector rows listed in rows[] (index k*Nv + v of proj) and
 * write them to out[r][Nu].  Cosine weight, then linear convolution along u
 * with the Ram-Lak kernel, zero outside the detector. */
int oracle_filter_rows(double R, int Nu, int Nv, int P, const float *proj,
                       long nrows, const long *rows, double *out) {
    if (R <= 0 || Nu <= 0 || Nv <= 0 || P <= 0 || nrows < 0) return ORACLE_EINVAL;
    int bad = 0;
#pragma omp parallel
    {
        double *q = (double *)malloc(sizeof(double) * (size_t)Nu);
        if (!q) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (long r = 0; r < nrows; ++r) {
            if (!q) continue;
            long row = rows[r];
            if (row < 0 || row >= (long)P * Nv) {
#pragma omp atomic write
                bad = 2;
                continue;
            }
            int v = (int)(row % Nv);
            double b = centre(v, Nv);
            const float *p = proj + (size_t)row * Nu;
            for (int m = 0; m < Nu; ++m) {
                double a = centre(m, Nu);
                q[m] = (double)p[m] * R / sqrt(R * R + a * a + b * b);
            }
            double *o = out + (size_t)r * Nu;
            for (int u = 0; u < Nu; ++u) {
                double acc = 0.0;
                for (int m = 0; m < Nu; ++m) acc += q[m] * ramlak((long)u - m);
                o[u] = acc;
            }
        }
        free(q);
    }
    return bad == 1 ? ORACLE_ENOMEM : (bad ? ORACLE_EINVAL : ORACLE_OK);
}

/* Filter every row: Q[P][Nv][Nu]. */
int oracle_filter(double R, int Nu, int Nv, int P, const float *proj, double *Q) {
    long n = (long)P * Nv;
    long *rows = (long *)malloc(sizeof(long) * (size_t)n);
    if (!rows) return ORACLE_ENOMEM;
    for (long r = 0; r < n; ++r) rows[r] = r;
    int rc = oracle_filter_rows(R, Nu, Nv, P, proj, n, rows, Q);
    free(rows);
    return rc;
}

/* ------------------------------------------------------- sample access */

/* Projection data is accepted as float32 (the values the GPU sees, exact in
 * FP64) or float64 (the oracle's own filter output). */
typedef struct {
    const void *p;
    int f64;
} qbuf;

static double qat(qbuf q, size_t i) {
    return q.f64 ? ((const double *)q.p)[i] : (double)((const float *)q.p)[i];
}

/* Bilinear sample of a [rows][cols] image at column c, row r; integer
 * positions outside the image contribute zero. */
static double bilerp(qbuf img, size_t off, int rows, int cols, double c, double r) {
    double c0 = floor(c), r0 = floor(r);
    double fc = c - c0, fr = r - r0;
    long ic = (long)c0, ir = (long)r0;
    double s[2][2];
    for (int dr = 0; dr < 2; ++dr)
        for (int dc = 0; dc < 2; ++dc) {
            long rr = ir + dr, cc = ic + dc;
            s[dr][dc] = (rr >= 0 && rr < rows && cc >= 0 && cc < cols)
                            ? qat(img, off + (size_t)rr * cols + (size_t)cc)
                            : 0.0;
        }
    return (1.0 - fr) * ((1.0 - fc) * s[0][0] + fc * s[0][1]) +
           fr * ((1.0 - fc) * s[1][0] + fc * s[1][1]);
}

/* ------------------------------------------------------------ plain FDK */

/* Plain FDK backprojection of the requested z-slices:
 * vol[iz][y][x] = (pi/P) sum_k U_k^-2 Q_k(u_k, v_k), u from Eq. 1,
 * v = z / U + (Nv-1)/2 (the row formula b of Sec. 2.2), summed in k order. */
static int fdk_slices(double R, int N, int Nu, int Nv, int P, qbuf Q, int nz,
                      const int *zs, double *vol) {
    if (R <= 0 || N <= 0 || Nu <= 0 || Nv <= 0 || P <= 0 || nz < 0) return ORACLE_EINVAL;
    for (int i = 0; i < nz; ++i)
        if (zs[i] < 0 || zs[i] >= N) return ORACLE_EINVAL;
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)P);
    if (!cs) return ORACLE_ENOMEM;
    for (int k = 0; k < P; ++k) {
        cs[2 * k] = cos(beta_of(k, P));
        cs[2 * k + 1] = sin(beta_of(k, P));
    }
    const double uc = 0.5 * (double)(Nu - 1), vc = 0.5 * (double)(Nv - 1);
    long lines = (long)nz * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (long l = 0; l < lines; ++l) {
        int iz = (int)(l / N), iy = (int)(l % N);
        double z = centre(zs[iz], N), y = centre(iy, N);
        for (int ix = 0; ix < N; ++ix) {
            double x = centre(ix, N);
            double acc = 0.0;
            for (int k = 0; k < P; ++k) {
                double cb = cs[2 * k], sb = cs[2 * k + 1];
                double u = eq1_a(R, x, y, cb, sb) + uc;
                double U = fdk_U(R, x, y, cb, sb);
                double v = z / U + vc;
                double val = bilerp(Q, (size_t)k * Nv * Nu, Nv, Nu, u, v);
                acc += val / (U * U);
            }
            vol[((size_t)iz * N + iy) * N + ix] = (M_PI / (double)P) * acc;
        }
    }
    free(cs);
    return ORACLE_OK;
}

int oracle_fdk_slices(double R, int N, int Nu, int Nv, int P, const void *Q, int q_f64,
                      int nz, const int *zs, double *vol) {
    qbuf q = {Q, q_f64};
    return fdk_slices(R, N, Nu, Nv, P, q, nz, zs, vol);
}

int oracle_fdk(double R, int N, int Nu, int Nv, int P, const void *Q, int q_f64, double *vol) {
    int *zs = (int *)malloc(sizeof(int) * (size_t)N);
    if (!zs) return ORACLE_ENOMEM;
    for (int i = 0; i < N; ++i) zs[i] = i;
    qbuf q = {Q, q_f64};
    int rc = fdk_slices(R, N, Nu, Nv, P, q, N, zs, vol);
    free(zs);
    return rc;
}

/* --------------------------------------------------------------- bounds */

/* Per square q = qy * 2^s + qx and angle k (Sec. 2.1, Eq. 1 at the square's
 * four vertices; Sec. 2.2 decomposition into 4^s squares):
 *   lo[q][k] = floor(min u), hi[q][k] = floor(max u) + 1 (columns read);
 *   phi[q][k] = a(x_c, y_c, beta_k) + (Nu-1)/2 (shift centre);
 *   w0[q] = floor(min_k (min u - phi)) - 1,
 *   T[q]  = floor(max_k (max u - phi)) + 3 - w0[q] (shifted-row width);
 *   crop[q][k] = floor(phi + w0) (first column the shifted row reads).
 * Any output pointer may be NULL. */
int oracle_bounds(double R, int N, int Nu, int P, int s, int32_t *lo, int32_t *hi,
                  int32_t *crop, double *phi, int32_t *w0, int32_t *T) {
    if (R <= 0 || N <= 0 || Nu <= 0 || P <= 0 || s < 0 || s > 20 || (1L << s) > N)
        return ORACLE_EINVAL;
    int m = 1 << s;
    long nsq = (long)m * m;
    const double uc = 0.5 * (double)(Nu - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (long q = 0; q < nsq; ++q) {
        int qy = (int)(q / m), qx = (int)(q % m);
        int ix0, ix1, iy0, iy1;
        square_range(qx, s, N, &ix0, &ix1);
        square_range(qy, s, N, &iy0, &iy1);
        double xs[2] = {centre(ix0, N), centre(ix1, N)};
        double ys[2] = {centre(iy0, N), centre(iy1, N)};
        double xc = 0.5 * (xs[0] + xs[1]), yc = 0.5 * (ys[0] + ys[1]);
        double dmin = INFINITY, dmax = -INFINITY;
        double *ph = (double *)malloc(sizeof(double) * (size_t)P);
        for (int k = 0; k < P; ++k) {
            double b = beta_of(k, P);
            double cb = cos(b), sb = sin(b);
            double umin = INFINITY, umax = -INFINITY;
            for (int vy = 0; vy < 2; ++vy)
                for (int vx = 0; vx < 2; ++vx) {
                    double u = eq1_a(R, xs[vx], ys[vy], cb, sb) + uc;
                    if (u < umin) umin = u;
                    if (u > umax) umax = u;
                }
            double p = eq1_a(R, xc, yc, cb, sb) + uc;
            ph[k] = p;
            if (lo) lo[q * P + k] = (int32_t)floor(umin);
            if (hi) hi[q * P + k] = (int32_t)floor(umax) + 1;
            if (phi) phi[q * P + k] = p;
            if (umin - p < dmin) dmin = umin - p;
            if (umax - p > dmax) dmax = umax - p;
        }
        int32_t w = (int32_t)floor(dmin) - 1;
        if (w0) w0[q] = w;
        if (T) T[q] = (int32_t)floor(dmax) + 3 - w;
        if (crop)
            for (int k = 0; k < P; ++k) crop[q * P + k] = (int32_t)floor(ph[k] + (double)w);
        free(ph);
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------ FDK-OD stages */

typedef struct {
    double R;
    int N, Nu, Nv, P, s, D, Pd;
    const double *h; /* angular taps h[|i|], |i| < H D; NULL: triangle */
    int H;
    int nsq;       /* 4^s */
    double *phi;   /* [nsq][P] */
    int32_t *lo, *hi, *w0, *T;
} odplan;

static void odplan_free(odplan *o) {
    free(o->phi);
    free(o->lo);
    free(o->hi);
    free(o->w0);
    free(o->T);
}

static int odplan_make(odplan *o, double R, int N, int Nu, int Nv, int P, int s, int D, const double *h,
                       int H) {
    memset(o, 0, sizeof(*o));
    if (D <= 0 || P <= 0 || P % D != 0) return ORACLE_EINVAL;
    if (H < 1 || (h == NULL && H != 1)) return ORACLE_EINVAL;
    o->h = h;
    o->H = H;
    if (s < 0 || s > 20 || (1L << s) > N) return ORACLE_EINVAL;
    o->R = R;
    o->N = N;
    o->Nu = Nu;
    o->Nv = Nv;
    o->P = P;
    o->s = s;
    o->D = D;
    o->Pd = P / D;
    o->nsq = (1 << s) * (1 << s);
    size_t n = (size_t)o->nsq * P;
    o->phi = (double *)malloc(sizeof(double) * n);
    o->lo = (int32_t *)malloc(sizeof(int32_t) * n);
    o->hi = (int32_t *)malloc(sizeof(int32_t) * n);
    o->w0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)o->nsq);
    o->T = (int32_t *)malloc(sizeof(int32_t) * (size_t)o->nsq);
    if (!o->phi || !o->lo || !o->hi || !o->w0 || !o->T) {
        odplan_free(o);
        return ORACLE_ENOMEM;
    }
    return oracle_bounds(R, N, Nu, P, s, o->lo, o->hi, NULL, o->phi, o->w0, o->T);
}

/* Linear interpolation of one detector row at column position pos, zero
 * outside the detector (Sec. 2.1: simple linear interpolation). */
static double lerp_row(qbuf Q, size_t off, int Nu, double pos) {
    double c0 = floor(pos);
    double f = pos - c0;
    long i = (long)c0;
    double a = (i >= 0 && i < Nu) ? qat(Q, off + (size_t)i) : 0.0;
    double b = (i + 1 >= 0 && i + 1 < Nu) ? qat(Q, off + (size_t)(i + 1)) : 0.0;
    return (1.0 - f) * a + f * b;
}

/* Shift then decimate one detector row v for square q (Sec. 2.1):
 *   1. shift: S[k][t] = Q_k(v, phi_k + w0 + t), t = 0..T-1, which puts the
 *      square centre on one column for every angle;
 *   2. low-pass along the angle axis: F[k][t] = sum_i h_i S[(k+i) mod P][t],
 *      h_i = (D - |i|) / D^2 for |i| < D (or the given taps, |i| < H D);
 *   3. downsample: S'[j][t] = F[j D][t], j = 0..P/D-1.
 * out[j][t] has row stride T (one row v only). */
static void shift_decimate_row(const odplan *o, qbuf Q, int q, int v, double *S, double *out) {
    int P = o->P, D = o->D, Nu = o->Nu, Nv = o->Nv, T = o->T[q], w0 = o->w0[q];
    for (int k = 0; k < P; ++k) {
        size_t off = ((size_t)k * Nv + v) * Nu;
        double p = o->phi[(size_t)q * P + k];
        for (int t = 0; t < T; ++t) S[(size_t)k * T + t] = lerp_row(Q, off, Nu, (p + (double)w0) + (double)t);
    }
    for (int j = 0; j < o->Pd; ++j) {
        for (int t = 0; t < T; ++t) {
            double acc = 0.0;
            int half = o->H * D;
            for (int i = -(half - 1); i <= half - 1; ++i) {
                int k = ((j * D + i) % P + P) % P;
                double h = o->h ? o->h[abs(i)] : (double)(D - abs(i)) / ((double)D * (double)D);
                acc += h * S[(size_t)k * T + t];
            }
            out[(size_t)j * T + t] = acc;
        }
    }
}

/* Decomposed data S'_q[j][v][t] of one square (all detector rows), for
 * inspecting the shift/decimation stage on its own.  D > 1 only. */
int oracle_shift_decimate(double R, int N, int Nu, int Nv, int P, int s, int D,
                          const void *Q, int q_f64, int q, double *out, const double *h, int H) {
    if (D < 2) return ORACLE_EINVAL;
    odplan o;
    int rc = odplan_make(&o, R, N, Nu, Nv, P, s, D, h, H);
    if (rc) return rc;
    if (q < 0 || q >= o.nsq) {
        odplan_free(&o);
        return ORACLE_EINVAL;
    }
    qbuf qb = {Q, q_f64};
    int T = o.T[q];
    int bad = 0;
#pragma omp parallel
    {
        double *S = (double *)malloc(sizeof(double) * (size_t)P * T);
        double *row = (double *)malloc(sizeof(double) * (size_t)o.Pd * T);
        if (!S || !row) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < Nv; ++v) {
            if (!S || !row) continue;
            shift_decimate_row(&o, qb, q, v, S, row);
            for (int j = 0; j < o.Pd; ++j)
                memcpy(out + ((size_t)j * Nv + v) * T, row + (size_t)j * T, sizeof(double) * T);
        }
        free(S);
        free(row);
    }
    odplan_free(&o);
    return bad ? ORACLE_ENOMEM : ORACLE_OK;
}

/* Sample position of voxel (x, y, z) in decimated view j of square q's
 * decomposed data (Sec. 2.2): column t = u - phi - w0 (the shift back folded
 * in), row v = z / U + (Nv-1)/2, and U (the weight is U^-2). */
static void od_sample_pos(const odplan *o, const double *cs, int q, int j, double x, double y, double z,
                          double *t, double *v, double *Uo) {
    int k = j * o->D;
    double cb = cs[2 * k], sb = cs[2 * k + 1];
    double u = eq1_a(o->R, x, y, cb, sb) + 0.5 * (double)(o->Nu - 1);
    double U = fdk_U(o->R, x, y, cb, sb);
    *t = u - o->phi[(size_t)q * o->P + k] - (double)o->w0[q];
    *v = z / U + 0.5 * (double)(o->Nv - 1);
    *Uo = U;
}

/* One voxel of square q backprojected from its decomposed data
 * sp[j][v][t] (j < P/D, Nv rows, T_q columns), scale pi / (P/D). */
static double bp_decomposed_voxel(const odplan *o, const double *cs, qbuf sp, int q, double x, double y,
                                  double z) {
    int T = o->T[q], Nv = o->Nv;
    double acc = 0.0;
    for (int j = 0; j < o->Pd; ++j) {
        double t, v, U;
        od_sample_pos(o, cs, q, j, x, y, z, &t, &v, &U);
        double val = bilerp(sp, (size_t)j * Nv * T, Nv, T, t, v);
        acc += val / (U * U);
    }
    return (M_PI / (double)o->Pd) * acc;
}

/* FDK-OD backprojection of the requested z-slices (Sec. 2.2):
 *   D = 1: each square reads its crop [lo, hi] of Q directly (no shift);
 *          every column read is checked against the crop window;
 *   D > 1: each square is backprojected from its decomposed data S'_q at
 *          the P/D angles beta_{jD}, with scale pi / (P/D) and column
 *          coordinate t = u - phi - w0 (the shift back folded in). */
int oracle_fdkod_slices(double R, int N, int Nu, int Nv, int P, int s, int D,
                        const void *Q, int q_f64, int nz, const int *zs, double *vol, const double *h, int H) {
    if (nz < 0) return ORACLE_EINVAL;
    for (int i = 0; i < nz; ++i)
        if (zs[i] < 0 || zs[i] >= N) return ORACLE_EINVAL;
    odplan o;
    int rc = odplan_make(&o, R, N, Nu, Nv, P, s, D, h, H);
    if (rc) return rc;
    qbuf qb = {Q, q_f64};
    const double uc = 0.5 * (double)(Nu - 1), vc = 0.5 * (double)(Nv - 1);
    int m = 1 << s, Pd = o.Pd;
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)P);
    if (!cs) {
        odplan_free(&o);
        return ORACLE_ENOMEM;
    }
    for (int k = 0; k < P; ++k) {
        cs[2 * k] = cos(beta_of(k, P));
        cs[2 * k + 1] = sin(beta_of(k, P));
    }
    /* detector rows any requested slice can touch: U lies in
     * [1 - r/R, 1 + r/R] with r the largest in-slice radius */
    char *need = (char *)calloc((size_t)Nv, 1);
    double rmax = sqrt(2.0) * 0.5 * (double)(N - 1);
    for (int i = 0; i < nz; ++i) {
        double z = centre(zs[i], N);
        double va = z / (1.0 - rmax / R) + vc, vb = z / (1.0 + rmax / R) + vc;
        double v0 = va < vb ? va : vb, v1 = va < vb ? vb : va;
        long r0 = (long)floor(v0) - 1, r1 = (long)floor(v1) + 2;
        for (long r = r0; r <= r1; ++r)
            if (r >= 0 && r < Nv) need[r] = 1;
    }
    int err = ORACLE_OK;
    for (int q = 0; q < o.nsq && err == ORACLE_OK; ++q) {
        int qy = q / m, qx = q % m;
        int ix0, ix1, iy0, iy1;
        square_range(qx, s, N, &ix0, &ix1);
        square_range(qy, s, N, &iy0, &iy1);
        int T = o.T[q];
        double *Sp = NULL;
        if (D > 1) {
            Sp = (double *)calloc((size_t)Pd * Nv * T, sizeof(double));
            if (!Sp) {
                err = ORACLE_ENOMEM;
                break;
            }
            int bad = 0;
#pragma omp parallel
            {
                double *S = (double *)malloc(sizeof(double) * (size_t)P * T);
                double *row = (double *)malloc(sizeof(double) * (size_t)Pd * T);
                if (!S || !row) {
#pragma omp atomic write
                    bad = 1;
                }
#pragma omp for schedule(dynamic, 1)
                for (int v = 0; v < Nv; ++v) {
                    if (!S || !row || !need[v]) continue;
                    shift_decimate_row(&o, qb, q, v, S, row);
                    for (int j = 0; j < Pd; ++j)
                        memcpy(Sp + ((size_t)j * Nv + v) * T, row + (size_t)j * T, sizeof(double) * T);
                }
                free(S);
                free(row);
            }
            if (bad) {
                free(Sp);
                err = ORACLE_ENOMEM;
                break;
            }
        }
        int crop_violation = 0;
        long lines = (long)nz * (iy1 - iy0 + 1);
        qbuf sp = {Sp, 1};
#pragma omp parallel for schedule(dynamic, 1)
        for (long l = 0; l < lines; ++l) {
            int iz = (int)(l / (iy1 - iy0 + 1)), iy = iy0 + (int)(l % (iy1 - iy0 + 1));
            double z = centre(zs[iz], N), y = centre(iy, N);
            for (int ix = ix0; ix <= ix1; ++ix) {
                double x = centre(ix, N);
                double acc = 0.0;
                if (D == 1) {
                    for (int k = 0; k < P; ++k) {
                        double cb = cs[2 * k], sb = cs[2 * k + 1];
                        double u = eq1_a(R, x, y, cb, sb) + uc;
                        double U = fdk_U(R, x, y, cb, sb);
                        double v = z / U + vc;
                        long c0 = (long)floor(u);
                        if (c0 < o.lo[(size_t)q * P + k] || c0 + 1 > o.hi[(size_t)q * P + k]) {
#pragma omp atomic write
                            crop_violation = 1;
                        }
                        double val = bilerp(qb, (size_t)k * Nv * Nu, Nv, Nu, u, v);
                        acc += val / (U * U);
                    }
                    vol[((size_t)iz * N + iy) * N + ix] = (M_PI / (double)P) * acc;
                } else {
                    vol[((size_t)iz * N + iy) * N + ix] = bp_decomposed_voxel(&o, cs, sp, q, x, y, z);
                }
            }
        }
        free(Sp);
        if (crop_violation) err = ORACLE_ECROP;
    }
    free(need);
    free(cs);
    odplan_free(&o);
    return err;
}

int oracle_fdkod(double R, int N, int Nu, int Nv, int P, int s, int D, const void *Q,
                 int q_f64, double *vol, const double *h, int H) {
    int *zs = (int *)malloc(sizeof(int) * (size_t)N);
    if (!zs) return ORACLE_ENOMEM;
    for (int i = 0; i < N; ++i) zs[i] = i;
    int rc = oracle_fdkod_slices(R, N, Nu, Nv, P, s, D, Q, q_f64, N, zs, vol, h, H);
    free(zs);
    return rc;
}

/* ------------------------------------- pieces for the learned decimation */

/* Step 1 of Sec. 2.1 alone: the shifted rows of square q at the full view
 * rate, S[k][v - v0][t] = Q_k(v, phi_k + w0 + t), t < T_q, for detector rows
 * v0 .. v0 + nv - 1 (the input of a learned angular low-pass). */
int oracle_shift_rows(double R, int N, int Nu, int Nv, int P, int s, const void *Q, int q_f64, int q, int v0,
                      int nv, double *out) {
    odplan o;
    int rc = odplan_make(&o, R, N, Nu, Nv, P, s, 1, NULL, 1);
    if (rc) return rc;
    if (q < 0 || q >= o.nsq || v0 < 0 || nv < 0 || v0 + nv > Nv) {
        odplan_free(&o);
        return ORACLE_EINVAL;
    }
    qbuf qb = {Q, q_f64};
    int T = o.T[q], w0 = o.w0[q];
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < P; ++k) {
        double p = o.phi[(size_t)q * P + k];
        for (int v = 0; v < nv; ++v) {
            size_t off = ((size_t)k * Nv + (size_t)(v0 + v)) * Nu;
            for (int t = 0; t < T; ++t)
                out[((size_t)k * nv + v) * T + t] = lerp_row(qb, off, Nu, (p + (double)w0) + (double)t);
        }
    }
    odplan_free(&o);
    return ORACLE_OK;
}

static double *trig_table(int P) {
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)P);
    if (!cs) return NULL;
    for (int k = 0; k < P; ++k) {
        cs[2 * k] = cos(beta_of(k, P));
        cs[2 * k + 1] = sin(beta_of(k, P));
    }
    return cs;
}

/* Backprojection of given decomposed data Sp[j][v][t] of square q (j < P/D,
 * all Nv rows, T_q columns) into the square's voxels on slices zs (Sec. 2.2,
 * the same sum as oracle_fdkod_slices); vol[nz][N][N], only square q's
 * voxels are written. */
int oracle_bp_square(double R, int N, int Nu, int Nv, int P, int s, int D, const double *Sp, int q, int nz,
                     const int *zs, double *vol) {
    for (int i = 0; i < nz; ++i)
        if (zs[i] < 0 || zs[i] >= N) return ORACLE_EINVAL;
    odplan o;
    int rc = odplan_make(&o, R, N, Nu, Nv, P, s, D, NULL, 1);
    if (rc) return rc;
    double *cs = trig_table(P);
    if (q < 0 || q >= o.nsq || !cs) {
        free(cs);
        odplan_free(&o);
        return cs ? ORACLE_EINVAL : ORACLE_ENOMEM;
    }
    int m = 1 << s, ix0, ix1, iy0, iy1;
    square_range(q % m, s, N, &ix0, &ix1);
    square_range(q / m, s, N, &iy0, &iy1);
    qbuf sp = {Sp, 1};
    long lines = (long)nz * (iy1 - iy0 + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (long l = 0; l < lines; ++l) {
        int iz = (int)(l / (iy1 - iy0 + 1)), iy = iy0 + (int)(l % (iy1 - iy0 + 1));
        double z = centre(zs[iz], N), y = centre(iy, N);
        for (int ix = ix0; ix <= ix1; ++ix)
            vol[((size_t)iz * N + iy) * N + ix] = bp_decomposed_voxel(&o, cs, sp, q, centre(ix, N), y, z);
    }
    free(cs);
    odplan_free(&o);
    return ORACLE_OK;
}

/* Adjoint of oracle_bp_square: dSp[j][v][t] = sum over square q's voxels on
 * slices zs of E[iz][y][x] times the weight with which sample (j, v, t)
 * enters that voxel, (pi / (P/D)) U^-2 times its bilinear weight (samples
 * outside [0, Nv) x [0, T_q) have none).  dSp is overwritten.  Serial: the
 * scatter sums in voxel order. */
int oracle_bp_square_adjoint(double R, int N, int Nu, int Nv, int P, int s, int D, const double *E, int q,
                             int nz, const int *zs, double *dSp) {
    for (int i = 0; i < nz; ++i)
        if (zs[i] < 0 || zs[i] >= N) return ORACLE_EINVAL;
    odplan o;
    int rc = odplan_make(&o, R, N, Nu, Nv, P, s, D, NULL, 1);
    if (rc) return rc;
    double *cs = trig_table(P);
    if (q < 0 || q >= o.nsq || !cs) {
        free(cs);
        odplan_free(&o);
        return cs ? ORACLE_EINVAL : ORACLE_ENOMEM;
    }
    int m = 1 << s, ix0, ix1, iy0, iy1, T = o.T[q];
    square_range(q % m, s, N, &ix0, &ix1);
    square_range(q / m, s, N, &iy0, &iy1);
    memset(dSp, 0, sizeof(double) * (size_t)o.Pd * Nv * T);
    double scale = M_PI / (double)o.Pd;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = iy0; iy <= iy1; ++iy)
            for (int ix = ix0; ix <= ix1; ++ix) {
                double e = E[((size_t)iz * N + iy) * N + ix];
                double x = centre(ix, N), y = centre(iy, N), z = centre(zs[iz], N);
                for (int j = 0; j < o.Pd; ++j) {
                    double t, v, U;
                    od_sample_pos(&o, cs, q, j, x, y, z, &t, &v, &U);
                    double c0 = floor(t), r0 = floor(v);
                    double fc = t - c0, fr = v - r0;
                    double g = scale * e / (U * U);
                    double wt[2][2] = {{(1.0 - fr) * (1.0 - fc), (1.0 - fr) * fc}, {fr * (1.0 - fc), fr * fc}};
                    for (int dr = 0; dr < 2; ++dr)
                        for (int dc = 0; dc < 2; ++dc) {
                            long rr = (long)r0 + dr, cc = (long)c0 + dc;
                            if (rr >= 0 && rr < Nv && cc >= 0 && cc < T)
                                dSp[((size_t)j * Nv + (size_t)rr) * T + (size_t)cc] += g * wt[dr][dc];
                        }
                }
            }
    free(cs);
    odplan_free(&o);
    return ORACLE_OK;
}
