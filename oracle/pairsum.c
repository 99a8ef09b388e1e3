/*
 * FP64 CPU oracle: smoothing functions and the four regularized layer
 * operators, written as plain double loops.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  The
 * product path (the CUDA library) shares no code, header or constant with it.
 *
 * Notation (Section 5): y = target point, x = source point, yhat = y - x,
 * r = |yhat|, rho = r / delta, n = outward unit normal of the porous body
 * at x, w = quadrature weight at x.
 *
 * Every operator loops over all ordered (target, source) pairs, including
 * the self pair; at r = 0 the smoothed kernels take their finite limits.
 * Targets are split over OpenMP threads; the source loop is sequential.
 */
#include <math.h>
#include <stdint.h>

#define PI_D 3.14159265358979323846
#define NSER 24   /* Taylor terms used for rho < RHO_SERIES */
#define RHO_SERIES 0.5

/*
 * The smoothing factors of Section 5.3:
 *   s_i(rho) = erf(rho) + (2/sqrt(pi)) * rho * Q_i(rho^2) * exp(-rho^2)
 * with
 *   Q_1(t) = -(2t - 5)/3,             Q_2(t) = (2t - 3)/3,
 *   Q_3(t) = -(4t^2 - 14t + 3)/3,     Q_4(t) = -(8t^3 - 36t^2 + 6t + 9)/9.
 * Coefficients q[i][m] of t^m in Q_i.
 */
static const double QCOEF[4][4] = {
    {5.0 / 3.0, -2.0 / 3.0, 0.0, 0.0},
    {-1.0, 2.0 / 3.0, 0.0, 0.0},
    {-1.0, 14.0 / 3.0, -4.0 / 3.0, 0.0},
    {-1.0, -6.0 / 9.0, 36.0 / 9.0, -8.0 / 9.0},
};
/* s_i behaves like rho^P_i as rho -> 0; the kernels need s_i / rho^P_i. */
static const int PPOW[4] = {1, 3, 3, 5};

/* Closed form of s_i (Section 5.3), i in 1..4. */
double ssdo_s_closed(int i, double rho) {
    const double *q = QCOEF[i - 1];
    double t = rho * rho;
    double poly = q[0] + t * (q[1] + t * (q[2] + t * q[3]));
    return erf(rho) + (2.0 / sqrt(PI_D)) * rho * poly * exp(-t);
}

/*
 * Taylor coefficient c_k of rho^(2k+1) in s_i(rho) * sqrt(pi)/2:
 *   erf part:  (-1)^k / (k! (2k+1))
 *   Gaussian part: sum_m q_m (-1)^(k-m) / (k-m)!
 */
static double series_coef(int i, int k) {
    const double *q = QCOEF[i - 1];
    double fact = 1.0;
    for (int j = 2; j <= k; ++j) fact *= j;
    double c = ((k % 2) ? -1.0 : 1.0) / (fact * (2 * k + 1));
    for (int m = 0; m <= 3 && m <= k; ++m) {
        double f = 1.0;
        for (int j = 2; j <= k - m; ++j) f *= j;
        c += q[m] * (((k - m) % 2) ? -1.0 : 1.0) / f;
    }
    return c;
}

/*
 * sigma_i(rho) = s_i(rho) / rho^P_i, the smooth even function the kernels use.
 * For rho < 0.5 the closed form cancels (its O(rho) terms cancel for
 * i = 2, 3, 4), so the Taylor series is summed instead, starting at the first
 * power that does not vanish identically.
 */
double ssdo_sigma(int i, double rho) {
    int p = PPOW[i - 1];
    if (rho >= RHO_SERIES) {
        double s = ssdo_s_closed(i, rho);
        double rp = rho;
        for (int j = 1; j < p; ++j) rp *= rho;
        return s / rp;
    }
    double t = rho * rho;
    int k0 = (p - 1) / 2;           /* lower coefficients are exactly zero */
    double sum = 0.0, tp = 1.0;
    for (int k = k0; k < k0 + NSER; ++k) {
        sum += series_coef(i, k) * tp;
        tp *= t;
    }
    return (2.0 / sqrt(PI_D)) * sum;
}

/* Exported for the pins: s_i(rho) through the same branch the kernels use. */
double ssdo_s(int i, double rho) {
    double v = ssdo_sigma(i, rho);
    for (int j = 0; j < PPOW[i - 1]; ++j) v *= rho;
    return v;
}

/*
 * Laplace single layer (Section 5.1 with the smoothed kernel of 5.3):
 *   (L g)(y_i) = sum_j w_j g_j G^delta(y_i, x_j),
 *   G^delta = -s_1(rho) / (4 pi r) = -sigma_1(rho) / (4 pi delta).
 * Layout: xyz is [3][n] (x row, y row, z row), likewise nrm.
 */
void ssdo_laplace_sl(int64_t nt, const double *ty, int64_t ns, const double *sx,
                     const double *w, double delta, const double *g, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nt; ++i) {
        double y0 = ty[i], y1 = ty[nt + i], y2 = ty[2 * nt + i];
        double acc = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double d0 = y0 - sx[j], d1 = y1 - sx[ns + j], d2 = y2 - sx[2 * ns + j];
            double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double G = -ssdo_sigma(1, r / delta) / (4.0 * PI_D * delta);
            acc += w[j] * g[j] * G;
        }
        out[i] = acc;
    }
}

/*
 * Laplace double layer with subtraction (eq. H_subtr), D^L = H - I/2:
 *   (D^L p)(y_i) = sum_j w_j [p_j - p_i] dG^delta/dn_x,
 *   dG^delta/dn_x = -(yhat . n_j) s_2(rho) / (4 pi r^3)
 *                 = -(yhat . n_j) sigma_2(rho) / (4 pi delta^3).
 * The sign follows the unsmoothed kernel of Section 5.1.
 * Targets coincide with sources (p_i is the density at target i).
 */
void ssdo_laplace_dl(int64_t n, const double *xyz, const double *nrm, const double *w,
                     double delta, const double *p, int64_t nrows, const int64_t *rows,
                     double *out) {
    /* rows == NULL: every target; otherwise out[k] is the value at target rows[k] */
    double d3 = delta * delta * delta;
    int64_t nt = rows ? nrows : n;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = rows ? rows[k] : k;
        double y0 = xyz[i], y1 = xyz[n + i], y2 = xyz[2 * n + i];
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double d0 = y0 - xyz[j], d1 = y1 - xyz[n + j], d2 = y2 - xyz[2 * n + j];
            double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double yn = d0 * nrm[j] + d1 * nrm[n + j] + d2 * nrm[2 * n + j];
            double K = -yn * ssdo_sigma(2, r / delta) / (4.0 * PI_D * d3);
            acc += w[j] * (p[j] - p[i]) * K;
        }
        out[k] = acc;
    }
}

/*
 * Stokes single layer (Section 5.2 with the smoothed Stokeslet of 5.3):
 *   (M f)(y_i) = 1/(8 pi mu) sum_j w_j S^delta(y_i, x_j) f_j,
 *   S^delta_ab = delta_ab s_1/r + yhat_a yhat_b s_3/r^3
 *              = delta_ab sigma_1/delta + yhat_a yhat_b sigma_3/delta^3.
 * f and out are [3][n].
 */
void ssdo_stokes_sl(int64_t nt, const double *ty, int64_t ns, const double *sx,
                    const double *w, double delta, double mu, const double *f,
                    double *out) {
    double d3 = delta * delta * delta;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nt; ++i) {
        double y0 = ty[i], y1 = ty[nt + i], y2 = ty[2 * nt + i];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double d0 = y0 - sx[j], d1 = y1 - sx[ns + j], d2 = y2 - sx[2 * ns + j];
            double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double rho = r / delta;
            double c1 = ssdo_sigma(1, rho) / delta;
            double c3 = ssdo_sigma(3, rho) / d3;
            double f0 = f[j], f1 = f[ns + j], f2 = f[2 * ns + j];
            double yf = d0 * f0 + d1 * f1 + d2 * f2;
            a0 += w[j] * (c1 * f0 + c3 * d0 * yf);
            a1 += w[j] * (c1 * f1 + c3 * d1 * yf);
            a2 += w[j] * (c1 * f2 + c3 * d2 * yf);
        }
        double s = 1.0 / (8.0 * PI_D * mu);
        out[i] = s * a0;
        out[nt + i] = s * a1;
        out[2 * nt + i] = s * a2;
    }
}

/*
 * Stokes double layer with subtraction (eq. K_subtr), D^S = K + I/2:
 *   (D^S u)(y_i)_b = -1/(8 pi) sum_j w_j [u_j - u_i]_a T^delta_abc n_c(x_j),
 *   T^delta_abc = -6 yhat_a yhat_b yhat_c s_4/r^5
 *               = -6 yhat_a yhat_b yhat_c sigma_4/delta^5,
 * i.e. (D^S u)(y_i) = 6/(8 pi) sum_j w_j ((u_j-u_i).yhat)(yhat.n_j) yhat sigma_4/delta^5.
 * n is the outward normal of the porous body (into the fluid).
 */
void ssdo_stokes_dl(int64_t n, const double *xyz, const double *nrm, const double *w,
                    double delta, const double *u, int64_t nrows, const int64_t *rows,
                    double *out) {
    /* rows == NULL: every target; otherwise column k of out ([3][nrows]) is target rows[k] */
    double d5 = delta * delta * delta * delta * delta;
    int64_t nt = rows ? nrows : n;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = rows ? rows[k] : k;
        double y0 = xyz[i], y1 = xyz[n + i], y2 = xyz[2 * n + i];
        double ui0 = u[i], ui1 = u[n + i], ui2 = u[2 * n + i];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double d0 = y0 - xyz[j], d1 = y1 - xyz[n + j], d2 = y2 - xyz[2 * n + j];
            double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double du0 = u[j] - ui0, du1 = u[n + j] - ui1, du2 = u[2 * n + j] - ui2;
            double uy = du0 * d0 + du1 * d1 + du2 * d2;
            double yn = d0 * nrm[j] + d1 * nrm[n + j] + d2 * nrm[2 * n + j];
            double T = -6.0 * ssdo_sigma(4, r / delta) / d5;   /* T_abc = T * yhat_a yhat_b yhat_c */
            /* -(1/8pi) * du_a * T yhat_a yhat_b yhat_c n_c */
            double c = -(1.0 / (8.0 * PI_D)) * w[j] * uy * T * yn;
            a0 += c * d0;
            a1 += c * d1;
            a2 += c * d2;
        }
        out[k] = a0;
        out[nt + k] = a1;
        out[2 * nt + k] = a2;
    }
}

/*
 * Dense matrix of one operator (for the discrete iteration matrix of eq.
 * A_mat, Section 6): out is (nc n) x (nc n), row-major, with the densities and
 * results in the component-major order of the functions above (entry (a, i)
 * at a n + i).  op: 0 = L, 1 = D^L, 2 = M, 3 = D^S.  Entry by entry the same
 * kernels as the matrix-free loops; the subtraction of the double layers
 * puts minus the row's off-diagonal sum on the diagonal (block).
 */
void ssdo_operator_matrix(int op, int64_t n, const double *xyz, const double *nrm, const double *w,
                          double delta, double mu, double *out) {
    int nc = (op >= 2) ? 3 : 1;
    int64_t m = nc * n;
    double d3 = delta * delta * delta, d5 = d3 * delta * delta;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double y0 = xyz[i], y1 = xyz[n + i], y2 = xyz[2 * n + i];
        double diag[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int64_t j = 0; j < n; ++j) {
            double d[3] = {y0 - xyz[j], y1 - xyz[n + j], y2 - xyz[2 * n + j]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double rho = r / delta;
            double yn = d[0] * nrm[j] + d[1] * nrm[n + j] + d[2] * nrm[2 * n + j];
            if (op == 0) {
                out[i * m + j] = w[j] * (-ssdo_sigma(1, rho) / (4.0 * PI_D * delta));
            } else if (op == 1) {
                double K = w[j] * (-yn * ssdo_sigma(2, rho) / (4.0 * PI_D * d3));
                out[i * m + j] = K;
                diag[0][0] -= K;
            } else if (op == 2) {
                double c1 = ssdo_sigma(1, rho) / delta, c3 = ssdo_sigma(3, rho) / d3;
                double s = w[j] / (8.0 * PI_D * mu);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        out[(a * n + i) * m + b * n + j] = s * ((a == b ? c1 : 0.0) + c3 * d[a] * d[b]);
            } else {
                double T = -6.0 * ssdo_sigma(4, rho) / d5;
                double c = -(1.0 / (8.0 * PI_D)) * w[j] * T * yn;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double v = c * d[a] * d[b];    /* row component a, density component b */
                        out[(a * n + i) * m + b * n + j] = v;
                        diag[a][b] -= v;
                    }
            }
        }
        if (op == 1) out[i * m + i] += diag[0][0];
        if (op == 3)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) out[(a * n + i) * m + b * n + i] += diag[a][b];
    }
}

/* Number of OpenMP threads the oracle's loops run on (reported by the baseline). */
int ssdo_num_threads(void) {
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}

/* Sets the OpenMP thread count of the oracle's loops, for the baseline's
 * single-thread and all-core timings (t <= 0 leaves it unchanged). */
void ssdo_set_threads(int t) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
