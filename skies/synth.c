/* Seeded-input support: latitude profiles of a band-limited sky for the test
 * and benchmark generators.  This is spherical-harmonic synthesis (the "S" of
 * Eq. synthesis), not part of the analysis method under test.
 *
 * For each order m and each north-hemisphere latitude x_r = cos(theta_r) it
 * evaluates
 *     F_m^{N}(theta_r) = sum_l a_lm Pbar_l^m(x_r) / sqrt(2 pi)
 *     F_m^{S}(theta_r) = sum_l a_lm Pbar_l^m(-x_r) / sqrt(2 pi)
 * for every map of a batch, using Pbar_l^m(-x) = (-1)^{l+m} Pbar_l^m(x).
 * Pbar is the orthonormal associated Legendre function (Condon-Shortley phase),
 * produced by the three-term recurrence in l; its starting value is carried as
 * a mantissa and a power-of-two exponent so that it does not underflow.
 *
 * alm   : [n_alm][nmaps][2]   packed m-major, idx(l,m) = m(2 lmax + 1 - m)/2 + l
 * x     : [nr]                cos(theta) of the north latitudes (x >= 0)
 * fnorth, fsouth : [nmaps][nr][lmax+1][2]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define T_EXP 200

static long idx_lm(int l, int m, int lmax) {
    return (long)m * (2L * lmax + 1 - m) / 2 + l;
}

void skies_profiles(int lmax, int nr, const double* x, int nmaps,
                    const double* alm, double* fnorth, double* fsouth) {
    const double inv_sqrt_2pi = 1.0 / sqrt(2.0 * M_PI);
    const double two_mT = ldexp(1.0, -T_EXP);
    const double two_T = ldexp(1.0, T_EXP);
    /* log2 of the Pbar_m^m constant, accumulated over m */
    double* log2c = (double*)malloc(sizeof(double) * (lmax + 1));
    log2c[0] = 0.5 * log2(0.5);
    for (int m = 1; m <= lmax; ++m)
        log2c[m] = log2c[m - 1] + 0.5 * log2((2.0 * m + 1.0) / (2.0 * m));
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * 4 * (size_t)nmaps);
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= lmax; ++m) {
            for (int r = 0; r < nr; ++r) {
                double xr = x[r];
                double st = sqrt((1.0 - xr) * (1.0 + xr));
                memset(acc, 0, sizeof(double) * 4 * (size_t)nmaps);
                double L;
                if (m == 0) L = log2c[0];
                else if (st <= 0.0) L = -INFINITY;
                else L = log2c[m] + m * log2(st);
                if (L > -1.0e6) {
                    int e = 0;
                    if (L < 0) e = -T_EXP * (int)ceil(-L / T_EXP);
                    double cur = ((m & 1) ? -1.0 : 1.0) * exp2(L - e);
                    double prev = 0.0;
                    for (int l = m; l <= lmax; ++l) {
                        if (l > m) {
                            double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                            double nxt;
                            if (l == m + 1) nxt = a * xr * cur;
                            else {
                                double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) /
                                                (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
                                nxt = a * (xr * cur - b * prev);
                            }
                            prev = cur;
                            cur = nxt;
                            if (e < 0 && fabs(cur) > two_T) {
                                cur *= two_mT;
                                prev *= two_mT;
                                e += T_EXP;
                            }
                        }
                        double v;
                        if (e == 0) v = cur;
                        else if (e == -T_EXP) v = cur * two_mT;
                        else continue;
                        const double* a_l = alm + 2 * (size_t)nmaps * idx_lm(l, m, lmax);
                        double* dst = acc + (((l + m) & 1) ? 2 * (size_t)nmaps : 0);
                        for (int b = 0; b < 2 * nmaps; ++b) dst[b] += a_l[b] * v;
                    }
                }
                for (int b = 0; b < nmaps; ++b) {
                    size_t o = (((size_t)b * nr + r) * (lmax + 1) + m) * 2;
                    for (int c = 0; c < 2; ++c) {
                        double s = acc[2 * b + c], an = acc[2 * nmaps + 2 * b + c];
                        fnorth[o + c] = (s + an) * inv_sqrt_2pi;
                        fsouth[o + c] = (s - an) * inv_sqrt_2pi;
                    }
                }
            }
        }
        free(acc);
    }
    free(log2c);
}
