/* Pairwise O(N^2) DDA matvec in plain C -- TEST INFRASTRUCTURE ONLY.
 *
 * Same definition as oracle/dda.py:pairwise_matvec, written as a double loop
 * so that row samples of multi-million-dipole targets and the timed CPU
 * baseline finish in seconds.  Nothing in the product path links this file.
 *
 *   (A P)_j = beta_j P_j + sum_{l != j} A(r_j - r_l) P_l
 *   A(r)    = e^{ik rho}/rho [ k^2 (rr - I) + (ik rho - 1)/rho^2 (3 rr - I) ]
 *
 * (the DDA system A P = E of the guide's eq. AP=E, off-diagonal blocks in the
 * Draine 1988 form).  Layout: r[3*j + a] positions (lattice units), beta and
 * P/Y complex interleaved: beta[2*j], P[6*j + 2*a] (re) / P[6*j + 2*a + 1] (im).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void row(int64_t n, const double *r, double kd, const double *beta,
                const double *P, int64_t j, double *y)
{
    double complex acc[3] = {0, 0, 0};
    const double xj = r[3 * j], yj = r[3 * j + 1], zj = r[3 * j + 2];
    const double k2 = kd * kd;
    for (int64_t l = 0; l < n; ++l) {
        if (l == j) continue;
        double d[3] = {xj - r[3 * l], yj - r[3 * l + 1], zj - r[3 * l + 2]};
        double rho = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double rh[3] = {d[0] / rho, d[1] / rho, d[2] / rho};
        double complex ph = cexp(I * kd * rho) / rho;
        double complex c1 = ph * k2;                                /* multiplies (rr - I)   */
        double complex c2 = ph * (I * kd * rho - 1.0) / (rho * rho);  /* multiplies (3rr - I) */
        double complex p[3];
        for (int a = 0; a < 3; ++a)
            p[a] = P[6 * l + 2 * a] + I * P[6 * l + 2 * a + 1];
        double complex rp = rh[0] * p[0] + rh[1] * p[1] + rh[2] * p[2];
        for (int a = 0; a < 3; ++a)
            acc[a] += c1 * (rh[a] * rp - p[a]) + c2 * (3.0 * rh[a] * rp - p[a]);
    }
    double complex b = beta[2 * j] + I * beta[2 * j + 1];
    for (int a = 0; a < 3; ++a) {
        double complex pj = P[6 * j + 2 * a] + I * P[6 * j + 2 * a + 1];
        double complex v = acc[a] + b * pj;
        y[2 * a] = creal(v);
        y[2 * a + 1] = cimag(v);
    }
}

/* Full matvec: Y[6*j + ...] for every j. Returns the number of threads used. */
int oracle_pairwise_matvec(int64_t n, const double *r, double kd, const double *beta,
                           const double *P, double *Y)
{
    int nthreads = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            nthreads = omp_get_num_threads();
#endif
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < n; ++j)
            row(n, r, kd, beta, P, j, Y + 6 * j);
    }
    return nthreads;
}

/* Selected rows only: Y[6*i + ...] = (A P)_{rows[i]}. */
int oracle_pairwise_rows(int64_t n, const double *r, double kd, const double *beta,
                         const double *P, int64_t nrows, const int64_t *rows, double *Y)
{
    int nthreads = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            nthreads = omp_get_num_threads();
#endif
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nrows; ++i)
            row(n, r, kd, beta, P, rows[i], Y + 6 * i);
    }
    return nthreads;
}

/* Scattered field at arbitrary points (near-field rows): for each point q,
 * E[6*q + ...] = -sum_{l: r_l != x_q} A(x_q - r_l) P_l, the field of every
 * dipole except one sitting on the point itself (oracle/dda.py:
 * scattered_field).  x[3*q + a] point positions. */
int oracle_field_points(int64_t n, const double *r, double kd, const double *P,
                        int64_t npts, const double *x, double *E)
{
    int nthreads = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            nthreads = omp_get_num_threads();
#endif
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < npts; ++q) {
            double complex acc[3] = {0, 0, 0};
            const double k2 = kd * kd;
            for (int64_t l = 0; l < n; ++l) {
                double d[3] = {x[3 * q] - r[3 * l], x[3 * q + 1] - r[3 * l + 1], x[3 * q + 2] - r[3 * l + 2]};
                if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) continue;
                double rho = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double rh[3] = {d[0] / rho, d[1] / rho, d[2] / rho};
                double complex ph = cexp(I * kd * rho) / rho;
                double complex c1 = ph * k2;
                double complex c2 = ph * (I * kd * rho - 1.0) / (rho * rho);
                double complex p[3];
                for (int a = 0; a < 3; ++a)
                    p[a] = P[6 * l + 2 * a] + I * P[6 * l + 2 * a + 1];
                double complex rp = rh[0] * p[0] + rh[1] * p[1] + rh[2] * p[2];
                for (int a = 0; a < 3; ++a)
                    acc[a] += c1 * (rh[a] * rp - p[a]) + c2 * (3.0 * rh[a] * rp - p[a]);
            }
            for (int a = 0; a < 3; ++a) {
                E[6 * q + 2 * a] = -creal(acc[a]);
                E[6 * q + 2 * a + 1] = -cimag(acc[a]);
            }
        }
    }
    return nthreads;
}
