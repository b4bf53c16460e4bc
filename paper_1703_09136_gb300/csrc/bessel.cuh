// Bessel and Hankel functions of integer order, FP64, host + device.
//
// Methods (all standard, written here from their definitions):
//  * J_n(x), n = 0..nmax: Miller's backward recurrence
//        J_{n-1} = (2n / x) J_n - J_{n+1}
//    from a start index well above max(nmax, x), normalised with the
//    Neumann addition identity  J_0 + 2 sum_{k>=1} J_{2k} = 1.
//  * Y_0, Y_1 from the same sequence through the Neumann series
//        Y_0 = (2/pi) (ln(x/2) + gamma) J_0 - (4/pi) sum_{k>=1} (-1)^k J_{2k} / k
//    and its derivative (Y_1 = -Y_0', J_0' = -J_1, J_m' = (J_{m-1} - J_{m+1}) / 2)
//        Y_1 = -(2/pi) J_0 / x + (2/pi) (ln(x/2) + gamma) J_1
//              + (2/pi) sum_{k>=1} (-1)^k (J_{2k-1} - J_{2k+1}) / k.
//  * for small x the ascending series of J_0, Y_0 (harmonic numbers H_k):
//        J_0 = sum (-1)^k (x^2/4)^k / (k!)^2,
//        Y_0 = (2/pi)(ln(x/2) + gamma) J_0 + (2/pi) sum_{k>=1} (-1)^{k+1} H_k (x^2/4)^k / (k!)^2.
//  * H_n = J_n + i Y_n for n >= 2 by forward recurrence of H (stable: the
//    Y part dominates once n exceeds x).
#pragma once

#include "common.cuh"

#define HFMM_EULER_GAMMA 0.57721566490153286061
#define HFMM_PI 3.14159265358979323846
#define HFMM_2_OVER_PI 0.63661977236758134308

// Start index of the backward recurrence (even).
HD int miller_start(double x, int nmax) {
    double n0 = fmax((double)nmax, x);
    int m = (int)(n0 + 20.0 + sqrt(160.0 * (n0 + 1.0)));
    return m + (m & 1);
}

// J[0..nmax] (J may be null), and J0, J1, Y0, Y1 for x > 0.
HD void bessel_miller(double x, int nmax, double* J, double* J0o, double* J1o,
                      double* Y0o, double* Y1o) {
    const int m = miller_start(x, nmax > 1 ? nmax : 1);
    const double BIG = 1e250, SMALL = 1e-250;
    double tp = 0.0;          // t_{j+1}
    double t = 1e-30;         // t_j (arbitrary scale)
    double norm = 0.0;        // t_0 + 2 sum t_{2k}
    double sy0 = 0.0;         // sum_{k>=1} (-1)^k t_{2k} / k
    double sy1 = 0.0;         // sum_{k>=1} (-1)^k (t_{2k-1} - t_{2k+1}) / k
    double t1 = 0.0;
    const double inv = 2.0 / x;
    if (J) for (int i = 0; i <= nmax; ++i) J[i] = 0.0;
    // t_m = tiny, t_{m+1} = 0; walk j = m .. 1 producing t_{j-1}
    for (int j = m; j >= 1; --j) {
        if ((j & 1) == 0) {
            int kk = j >> 1;
            norm += 2.0 * t;
            double sgn = (kk & 1) ? -1.0 : 1.0;
            sy0 += sgn * t / (double)kk;
        } else {
            // odd j = 2k-1 with k = (j+1)/2 contributes +t_j; odd j = 2k+1 with k = (j-1)/2 contributes -t_j
            int ka = (j + 1) >> 1;
            double sa = (ka & 1) ? -1.0 : 1.0;
            sy1 += sa * t / (double)ka;
            int kb = (j - 1) >> 1;
            if (kb >= 1) {
                double sb = (kb & 1) ? -1.0 : 1.0;
                sy1 -= sb * t / (double)kb;
            }
        }
        if (J && j <= nmax) J[j] = t;
        if (j == 1) t1 = t;
        double tm = (double)j * inv * t - tp;
        tp = t;
        t = tm;
        if (fabs(t) > BIG) {
            t *= SMALL; tp *= SMALL; norm *= SMALL; sy0 *= SMALL; sy1 *= SMALL; t1 *= SMALL;
            if (J) for (int i = j; i <= nmax; ++i) J[i] *= SMALL;
        }
    }
    // t is t_0
    norm += t;
    const double s = 1.0 / norm;
    const double j0 = t * s, j1 = t1 * s;
    if (J) { J[0] = t; for (int i = 0; i <= nmax; ++i) J[i] *= s; }
    const double lg = log(0.5 * x) + HFMM_EULER_GAMMA;
    if (J0o) *J0o = j0;
    if (J1o) *J1o = j1;
    if (Y0o) *Y0o = HFMM_2_OVER_PI * (lg * j0 - 2.0 * sy0 * s);
    if (Y1o) *Y1o = HFMM_2_OVER_PI * (-j0 / x + lg * j1 + sy1 * s);
}

// Ascending series of J0 and Y0 (x <= 5).
HD void bessel_01_series(double x, double* J0o, double* Y0o) {
    const double q = 0.25 * x * x;
    double term = 1.0, j0 = 1.0, ys = 0.0, hk = 0.0;
    for (int k = 1; k < 40; ++k) {
        term *= -q / ((double)k * (double)k);
        hk += 1.0 / (double)k;
        j0 += term;
        ys -= hk * term;
        if (fabs(term) * (hk + 1.0) < 1e-18 * fabs(j0) + 1e-300) break;
    }
    *J0o = j0;
    *Y0o = HFMM_2_OVER_PI * ((log(0.5 * x) + HFMM_EULER_GAMMA) * j0 + ys);
}

// H_0^(1)(x) for x > 0.
HD cd hankel0(double x) {
    double j0, y0;
    if (x <= 5.0) {
        bessel_01_series(x, &j0, &y0);
    } else {
        bessel_miller(x, 1, nullptr, &j0, nullptr, &y0, nullptr);
    }
    return cmk(j0, y0);
}

// H_0 and H_1 for x > 0.
HD void hankel01(double x, cd* h0, cd* h1) {
    double j0, j1, y0, y1;
    bessel_miller(x, 1, nullptr, &j0, &j1, &y0, &y1);
    *h0 = cmk(j0, y0);
    *h1 = cmk(j1, y1);
}

// H[0..nmax] = H_n^(1)(x), x > 0, by forward recurrence from H_0, H_1.
HD void hankel_seq(double x, int nmax, cd* H) {
    cd h0, h1;
    hankel01(x, &h0, &h1);
    H[0] = h0;
    if (nmax >= 1) H[1] = h1;
    const double inv = 2.0 / x;
    for (int n = 1; n < nmax; ++n) {
        H[n + 1] = csub(cscale(H[n], (double)n * inv), H[n - 1]);
    }
}

// J[0..nmax] = J_n(x), x >= 0.
HD void bessel_j_seq(double x, int nmax, double* J) {
    if (x <= 0.0) {
        J[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) J[n] = 0.0;
        return;
    }
    bessel_miller(x, nmax, J, nullptr, nullptr, nullptr, nullptr);
}
