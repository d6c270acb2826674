/*
 * das_oracle.c -- plain FP64 CPU reference for volumetric delay-and-sum.
 *
 * TEST INFRASTRUCTURE ONLY (see das_oracle.h).  Written to be read against the
 * paper, not to be fast: every term of Eq. 2 is evaluated from its definition,
 * in the order the sums are written (q outer, m inner), with no tiling, no
 * reordering and no precomputed tables.  OpenMP only splits independent output
 * values (voxels, or channel rows for the adjoint) across threads; the order
 * of the additions into any single output value is fixed and sequential.
 *
 * Readings of the paper used here (the paper leaves these points open):
 *   R1 sample time origin: 0-based k, sample k is taken at t = k / fs, so a
 *      delay tau (seconds) sits at fractional index tau*fs.
 *   R2 receive delay ||p - r_m|| / c (Eq. 1, as printed).
 *   R3 diverging wave: tau^tx = (||p - v_q|| - ||v_q - o||) / c, i.e. t = 0 when
 *      the wave front passes the reference point o (the array centre); with
 *      t0_offset = 0 the paper's footnote form ||p - v_q|| / c is used.
 *   R4 plane wave: tau^tx = d_q . (p - o) / c with d_q the unit propagation
 *      direction (the footnote's minus sign reads as d pointing back at the
 *      array).  Photoacoustic (Sec. 2): tau^tx = 0.
 *   R5 IQ data: the focused sample is y[tau] * e^{+i 2 pi f_d tau}, which makes
 *      baseband data of a point reflector add in phase (IQ = 2 LPF{rf e^{-i 2 pi f_d t}}).
 *   R6 receive weight (Sec. 2, w^rx computed from element origin and direction):
 *      with e = p - r_m, z = e . n_m and rho^2 = |e|^2 - z^2, w^rx = 1 when the
 *      f-number is <= 0 (full aperture) or when z > 0 and
 *      rho^2 <= (1 + 1e-6) (z / (2 F))^2; otherwise 0.
 *   R7 out of range: a term contributes only when 0 <= k <= K - 2.
 *   R8 transmit weight w^tx: the table given, or 1.
 */
#include "das_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define APERTURE_MARGIN 1e-6

static long n_voxels(const das_oracle_problem *P)
{
    return (long)P->nx * P->ny * P->nz;
}

/* Voxel position on the grid (Sec. 2: p_n on an Nx x Ny x Nz grid). */
static void voxel_position(const das_oracle_problem *P, long n, double p[3])
{
    long ix = n % P->nx;
    long iy = (n / P->nx) % P->ny;
    long iz = n / ((long)P->nx * P->ny);
    p[0] = P->origin[0] + (double)ix * P->spacing[0];
    p[1] = P->origin[1] + (double)iy * P->spacing[1];
    p[2] = P->origin[2] + (double)iz * P->spacing[2];
}

static double dist3(const double a[3], const double b[3])
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Transmit delay tau^tx_qn in seconds (Eq. 1 and its footnote; readings R3, R4). */
static double transmit_delay(const das_oracle_problem *P, int q, const double p[3])
{
    const double *v = P->tx_vec + 3 * q;
    switch (P->tx_kind[q]) {
    case ORACLE_TX_DIVERGING: {
        double path = dist3(p, v);
        if (P->t0_offset) path -= dist3(v, P->t0_ref);
        return path / P->c;
    }
    case ORACLE_TX_PLANE:
        return (v[0] * (p[0] - P->t0_ref[0]) + v[1] * (p[1] - P->t0_ref[1]) +
                v[2] * (p[2] - P->t0_ref[2])) / P->c;
    default:
        return 0.0;
    }
}

/* Receive delay tau^rx_mn in seconds (Eq. 1). */
static double receive_delay(const das_oracle_problem *P, int m, const double p[3])
{
    return dist3(p, P->elem_pos + 3 * m) / P->c;
}

/* Receive weight w^rx_mn (Sec. 2, reading R6). */
static double receive_weight(const das_oracle_problem *P, int m, const double p[3])
{
    if (P->f_number <= 0.0) return 1.0;
    const double *r = P->elem_pos + 3 * m;
    const double *nrm = P->elem_normal + 3 * m;
    double e[3] = {p[0] - r[0], p[1] - r[1], p[2] - r[2]};
    double z = e[0] * nrm[0] + e[1] * nrm[1] + e[2] * nrm[2];
    if (!(z > 0.0)) return 0.0;
    double rho2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] - z * z;
    double half_width = z / (2.0 * P->f_number);
    return (rho2 <= (1.0 + APERTURE_MARGIN) * half_width * half_width) ? 1.0 : 0.0;
}

/* Transmit weight w^tx_qn (Sec. 2; reading R8). */
static double transmit_weight(const das_oracle_problem *P, int q, long n)
{
    return P->w_tx ? P->w_tx[(long)q * n_voxels(P) + n] : 1.0;
}

/* One term of Eq. 2: delay in samples, weight, and whether it contributes.
 * Returns 1 and fills (k, alpha, tau_s, w) when the term contributes. */
static int term(const das_oracle_problem *P, int q, int m, long n, const double p[3],
                long *k, double *alpha, double *tau_s, double *w)
{
    double wr = receive_weight(P, m, p);
    if (wr == 0.0) return 0;
    double tau = transmit_delay(P, q, p) + receive_delay(P, m, p); /* Eq. 1 */
    double ts = tau * P->fs;                                       /* R1 */
    double kf = floor(ts);
    if (kf < 0.0 || kf > (double)(P->K - 2)) return 0;             /* R7 */
    *k = (long)kf;
    *alpha = ts - kf;
    *tau_s = ts;
    *w = transmit_weight(P, q, n) * wr;
    return 1;
}

/* Channel sample y_bqm[k] widened to double (complex; imaginary part 0 for RF). */
static void sample(const das_oracle_problem *P, const void *y, int is_f64, int b, int q, int m,
                   long k, double *re, double *im)
{
    size_t idx = (((size_t)b * P->Q + q) * P->M + m) * (size_t)P->K + (size_t)k;
    if (is_f64) {
        const double *d = (const double *)y;
        if (P->iq) { *re = d[2 * idx]; *im = d[2 * idx + 1]; }
        else { *re = d[idx]; *im = 0.0; }
    } else {
        const float *f = (const float *)y;
        if (P->iq) { *re = (double)f[2 * idx]; *im = (double)f[2 * idx + 1]; }
        else { *re = (double)f[idx]; *im = 0.0; }
    }
}

/* Eq. 2 with linear interpolation (Sec. 2) and the IQ phase factor (R5). */
static void forward_impl(const das_oracle_problem *P, const void *y, int is_f64, int B,
                         const long *voxels, long nv, double *x)
{
    long N = n_voxels(P);
    if (!voxels) nv = N;
    double two_pi_fd_over_fs = 2.0 * M_PI * P->f_demod / P->fs;

#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < nv; ++i) {
        long n = voxels ? voxels[i] : i;
        double p[3];
        voxel_position(P, n, p);
        double *acc = (double *)calloc(2 * (size_t)B, sizeof(double));
        for (int q = 0; q < P->Q; ++q) {
            for (int m = 0; m < P->M; ++m) {
                long k;
                double alpha, ts, w;
                if (!term(P, q, m, n, p, &k, &alpha, &ts, &w)) continue;
                double ph = two_pi_fd_over_fs * ts;
                double cph = cos(ph), sph = sin(ph);
                for (int b = 0; b < B; ++b) {
                    double r0, i0, r1, i1;
                    sample(P, y, is_f64, b, q, m, k, &r0, &i0);
                    sample(P, y, is_f64, b, q, m, k + 1, &r1, &i1);
                    double sr = (1.0 - alpha) * r0 + alpha * r1;
                    double si = (1.0 - alpha) * i0 + alpha * i1;
                    acc[2 * b] += w * (sr * cph - si * sph);
                    acc[2 * b + 1] += w * (sr * sph + si * cph);
                }
            }
        }
        for (int b = 0; b < B; ++b) {
            x[2 * ((size_t)b * nv + i)] = acc[2 * b];
            x[2 * ((size_t)b * nv + i) + 1] = acc[2 * b + 1];
        }
        free(acc);
    }
}

void oracle_forward(const das_oracle_problem *P, const float *y, int B, const long *voxels,
                    long nv, double *x)
{
    forward_impl(P, y, 0, B, voxels, nv, x);
}

void oracle_forward_f64(const das_oracle_problem *P, const double *y, int B, const long *voxels,
                        long nv, double *x)
{
    forward_impl(P, y, 1, B, voxels, nv, x);
}

/* Adjoint of Eq. 2: each forward term w e^{i phi} ((1-a) y[k] + a y[k+1]) sends
 * conj(w e^{i phi}) (1-a) x_n to y[k] and conj(w e^{i phi}) a x_n to y[k+1].
 * Parallel over channel rows (q, m); within a row voxels are visited in order. */
void oracle_adjoint(const das_oracle_problem *P, const double *x, int B, const long *rows,
                    long nrows, double *y)
{
    long N = n_voxels(P);
    if (!rows) nrows = (long)P->Q * P->M;
    double two_pi_fd_over_fs = 2.0 * M_PI * P->f_demod / P->fs;
    memset(y, 0, sizeof(double) * 2 * (size_t)B * (size_t)nrows * P->K);

#pragma omp parallel for schedule(dynamic, 4)
    for (long j = 0; j < nrows; ++j) {
        long row_id = rows ? rows[j] : j;
        int q = (int)(row_id / P->M), m = (int)(row_id % P->M);
        for (long n = 0; n < N; ++n) {
            double p[3];
            voxel_position(P, n, p);
            long k;
            double alpha, ts, w;
            if (!term(P, q, m, n, p, &k, &alpha, &ts, &w)) continue;
            double ph = two_pi_fd_over_fs * ts;
            double cr = w * cos(ph), ci = -w * sin(ph); /* conj(w e^{i phi}) */
            for (int b = 0; b < B; ++b) {
                double xr = x[2 * ((size_t)b * N + n)], xi = x[2 * ((size_t)b * N + n) + 1];
                double vr = cr * xr - ci * xi, vi = cr * xi + ci * xr;
                size_t row = ((size_t)b * nrows + j) * (size_t)P->K;
                y[2 * (row + k)] += (1.0 - alpha) * vr;
                y[2 * (row + k) + 1] += (1.0 - alpha) * vi;
                y[2 * (row + k + 1)] += alpha * vr;
                y[2 * (row + k + 1) + 1] += alpha * vi;
            }
        }
    }
}

/* d x_bn / d c.  tau_s = fs * (path length) / c, so d tau_s / dc = -tau_s / c.
 * Within the interpolation cell [k, k+1] the interpolant has slope y[k+1] - y[k]
 * (the one-sided derivative at a sample), and d/dtau_s e^{i theta tau_s} =
 * i theta e^{i theta tau_s} with theta = 2 pi f_d / fs.  The aperture and
 * transmit weights do not depend on c. */
double oracle_grad_c(const das_oracle_problem *P, const float *y, const double *gx, int B,
                     const long *voxels, long nv)
{
    if (!voxels) nv = n_voxels(P);
    double theta = 2.0 * M_PI * P->f_demod / P->fs;
    double total = 0.0;

#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (long i = 0; i < nv; ++i) {
        long n = voxels ? voxels[i] : i;
        double p[3];
        voxel_position(P, n, p);
        double *dx = (double *)calloc(2 * (size_t)B, sizeof(double));
        for (int q = 0; q < P->Q; ++q) {
            for (int m = 0; m < P->M; ++m) {
                long k;
                double alpha, ts, w;
                if (!term(P, q, m, n, p, &k, &alpha, &ts, &w)) continue;
                double ph = theta * ts;
                double cph = cos(ph), sph = sin(ph);
                double dts = -ts / P->c;
                for (int b = 0; b < B; ++b) {
                    double r0, i0, r1, i1;
                    sample(P, y, 0, b, q, m, k, &r0, &i0);
                    sample(P, y, 0, b, q, m, k + 1, &r1, &i1);
                    double sr = (1.0 - alpha) * r0 + alpha * r1;
                    double si = (1.0 - alpha) * i0 + alpha * i1;
                    /* d/dtau_s of the interpolated, rotated sample, before the phase: */
                    double gr = (r1 - r0) - theta * si; /* slope + i*theta*s, real part */
                    double gi = (i1 - i0) + theta * sr; /* imaginary part */
                    dx[2 * b] += w * dts * (gr * cph - gi * sph);
                    dx[2 * b + 1] += w * dts * (gr * sph + gi * cph);
                }
            }
        }
        for (int b = 0; b < B; ++b) {
            double ar = gx[2 * ((size_t)b * nv + i)], ai = gx[2 * ((size_t)b * nv + i) + 1];
            total += ar * dx[2 * b] + ai * dx[2 * b + 1]; /* Re(conj(gx) * dx) */
        }
        free(dx);
    }
    return total;
}

long long oracle_count_active(const das_oracle_problem *P)
{
    long N = n_voxels(P);
    long long count = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : count)
    for (long n = 0; n < N; ++n) {
        double p[3];
        voxel_position(P, n, p);
        for (int q = 0; q < P->Q; ++q)
            for (int m = 0; m < P->M; ++m) {
                long k;
                double alpha, ts, w;
                if (term(P, q, m, n, p, &k, &alpha, &ts, &w)) ++count;
            }
    }
    return count;
}

long long oracle_count_near_ties(const das_oracle_problem *P, double rel)
{
    /* Counts pairs whose rho^2 lies within rel (relative) of the unshifted
     * threshold (z / 2F)^2 without being an exact tie (closer than 1e-9).
     * Exact ties fall inside the 1e-6 margin of reading R6 in any precision
     * near double's; pairs counted here are the ones whose decision could
     * flip between a float32 and a float64 evaluation. */
    if (P->f_number <= 0.0) return 0;
    long N = n_voxels(P);
    long long count = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : count)
    for (long n = 0; n < N; ++n) {
        double p[3];
        voxel_position(P, n, p);
        for (int m = 0; m < P->M; ++m) {
            const double *r = P->elem_pos + 3 * m;
            const double *nrm = P->elem_normal + 3 * m;
            double e[3] = {p[0] - r[0], p[1] - r[1], p[2] - r[2]};
            double z = e[0] * nrm[0] + e[1] * nrm[1] + e[2] * nrm[2];
            if (!(z > 0.0)) continue;
            double rho2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] - z * z;
            double hw = z / (2.0 * P->f_number);
            double thr = hw * hw;
            double d = fabs(rho2 - thr);
            if (d > 1e-9 * thr && d <= rel * thr) ++count;
        }
    }
    return count;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
