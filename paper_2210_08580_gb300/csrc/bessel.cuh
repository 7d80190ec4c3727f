// Bessel functions J0, Y0, J1, Y1 of real positive argument in FP64 for the kernel
// g2(r) = (i/4) H0^(1)(k r) of Sec. II and its normal derivative (H1^(1)).
//
// Written from the textbook representations (DLMF chapter 10), not from any library:
//   z <= 4        ascending power series (DLMF 10.2.2 for J, 10.8.1/10.8.2 for Y),
//                 all four functions from shared powers of z^2/4;
//   4 < z <= 30   Miller's backward recurrence J_{n-1} = (2n/z) J_n - J_{n+1} normalised
//                 by J0 + 2 sum J_2k = 1 (DLMF 10.12.4), Y0 from Neumann's expansion
//                 Y0 = (2/pi)(ln(z/2)+gamma) J0 - (4/pi) sum (-1)^k J_2k / k
//                 (Abramowitz & Stegun 9.1.88) and Y1 = -Y0' from its term-by-term
//                 derivative (J_2k' = (J_{2k-1} - J_{2k+1})/2);
//   z > 30        Hankel's asymptotic expansion (DLMF 10.17.3) to ~1e-17.
// Accuracy target: absolute error <= ~1e-15 (the Galerkin integrals need absolute, not
// relative, accuracy of g2).
#pragma once

#include <math.h>

#ifndef BEM_PI
#define BEM_PI 3.14159265358979323846
#endif
#define BEM_EULER_GAMMA 0.57721566490153286061

struct Bessel01 { double J0, Y0, J1, Y1; };

// Power series: q = z^2/4.
//   J0 = sum t_m,                t_m = (-q)^m/(m!)^2
//   Y0 = (2/pi)(ln(z/2)+g) J0 - (2/pi) sum_{m>=1} H_m t_m
//   J1 = (z/2) sum u_m,          u_m = (-q)^m/(m!(m+1)!)
//   Y1 = -2/(pi z) + (2/pi)(ln(z/2)+g) J1 - (z/(2 pi)) sum (H_m + H_{m+1}) u_m
template <bool WITH1>
__device__ __forceinline__ void bessel_series(double z, Bessel01& b) {
    const double q = 0.25 * z * z;
    double t = 1.0, u = 1.0, Hm = 0.0;
    double sJ0 = 1.0, sY0 = 0.0, sJ1 = 1.0, sY1 = 1.0;   // sY1 starts with (H_0 + H_1) u_0 = 1
    #pragma unroll 1
    for (int m = 1; m < 40; ++m) {
        const double dm = (double)m;
        t *= -q / (dm * dm);
        Hm += 1.0 / dm;
        sJ0 += t;
        sY0 += Hm * t;
        if (WITH1) {
            u *= -q / (dm * (dm + 1.0));
            sJ1 += u;
            sY1 += (2.0 * Hm + 1.0 / (dm + 1.0)) * u;
        }
        if (fabs(t) < 1e-18 && (!WITH1 || fabs(u) < 1e-18)) break;
    }
    const double lg = log(0.5 * z) + BEM_EULER_GAMMA;
    b.J0 = sJ0;
    b.Y0 = (2.0 / BEM_PI) * (lg * sJ0 - sY0);
    if (WITH1) {
        b.J1 = 0.5 * z * sJ1;
        b.Y1 = -2.0 / (BEM_PI * z) + (2.0 / BEM_PI) * lg * b.J1 - (z / (2.0 * BEM_PI)) * sY1;
    }
}

// Miller backward recurrence with Neumann series for Y0, Y1 (4 < z <= 30).  The start
// index z + 16 + 6 z^(1/3) puts J_nstart below 1e-17 of the normalisation.
template <bool WITH1>
__device__ __forceinline__ void bessel_miller(double z, Bessel01& b) {
    int nstart = 2 * (int)((z + 16.0 + 6.0 * cbrt(z)) * 0.5);
    double jp1 = 0.0, jn = 1e-30;         // J_{n+1}, J_n  (unnormalised)
    double norm = 0.0, neu0 = 0.0, neu1 = 0.0;
    double j_odd_above = 0.0;             // J_{2k+1} seen before J_{2k-1}
    const double iz2 = 2.0 / z;
    // loop invariant: at the top, jn = J_n, jp1 = J_{n+1}
    #pragma unroll 1
    for (int n = nstart; n >= 1; --n) {
        if ((n & 1) == 0) {
            const int kk = n >> 1;
            norm += 2.0 * jn;
            const double sgn = (kk & 1) ? -1.0 : 1.0;
            neu0 += sgn * jn / (double)kk;
            // (J_{2k-1} - J_{2k+1}) / k needs J_{2k-1}, obtained next step; keep J_{2k+1}
            j_odd_above = jp1;
        } else {
            // n = 2k - 1 with k = (n+1)/2: J_{2k-1} = jn, J_{2k+1} = j_odd_above
            const int kk = (n + 1) >> 1;
            const double sgn = (kk & 1) ? -1.0 : 1.0;
            neu1 += sgn * (jn - j_odd_above) / (double)kk;
        }
        const double jm1 = (double)n * iz2 * jn - jp1;
        jp1 = jn;
        jn = jm1;
        if (fabs(jn) > 1e250) {           // rescale to stay in range
            jn *= 1e-250; jp1 *= 1e-250; norm *= 1e-250; neu0 *= 1e-250; neu1 *= 1e-250;
            j_odd_above *= 1e-250;
        }
    }
    // now jn = J_0, jp1 = J_1 (unnormalised)
    norm += jn;
    const double s = 1.0 / norm;
    const double J0 = jn * s, J1 = jp1 * s;
    const double lg = log(0.5 * z) + BEM_EULER_GAMMA;
    b.J0 = J0;
    b.Y0 = (2.0 / BEM_PI) * lg * J0 - (4.0 / BEM_PI) * neu0 * s;
    if (WITH1) {
        b.J1 = J1;
        // Y1 = -Y0' = -(2/pi) J0/z + (2/pi)(ln(z/2)+g) J1 + (2/pi) sum (-1)^k (J_{2k-1}-J_{2k+1})/k
        b.Y1 = -(2.0 / BEM_PI) * J0 / z + (2.0 / BEM_PI) * lg * J1 + (2.0 / BEM_PI) * neu1 * s;
    }
}

// Hankel asymptotic expansion: H_nu(z) ~ sqrt(2/(pi z)) e^{i w} sum_k i^k a_k(nu) / z^k,
// w = z - nu pi/2 - pi/4, a_k = a_{k-1} (4 nu^2 - (2k-1)^2) / (8 k).
__device__ __forceinline__ void hankel_asym(double z, double nu, double& J, double& Y) {
    const double mu = 4.0 * nu * nu;
    double ak = 1.0, zk = 1.0;
    double sre = 1.0, sim = 0.0;          // sum i^k a_k / z^k
    #pragma unroll 1
    for (int k = 1; k < 30; ++k) {
        const double tk = (double)(2 * k - 1);
        ak *= (mu - tk * tk) / (8.0 * (double)k);
        zk /= z;
        const double term = ak * zk;
        switch (k & 3) {
            case 0: sre += term; break;
            case 1: sim += term; break;
            case 2: sre -= term; break;
            default: sim -= term; break;
        }
        if (fabs(term) < 1e-18) break;
    }
    const double w = z - (0.5 * nu + 0.25) * BEM_PI;
    double sw, cw;
    sincos(w, &sw, &cw);
    const double amp = sqrt(2.0 / (BEM_PI * z));
    J = amp * (cw * sre - sw * sim);
    Y = amp * (sw * sre + cw * sim);
}

template <bool WITH1>
__device__ __forceinline__ Bessel01 bessel01(double z) {
    Bessel01 b;
    if (z <= 4.0) {
        bessel_series<WITH1>(z, b);
    } else if (z <= 30.0) {
        bessel_miller<WITH1>(z, b);
    } else {
        hankel_asym(z, 0.0, b.J0, b.Y0);
        if (WITH1) hankel_asym(z, 1.0, b.J1, b.Y1);
    }
    return b;
}

// ---------------------------------------------------------------------------------------
// Table-driven evaluation for the far field, as polynomials in u = z^2: no square root, no
// logarithm and (for S, N) no division on the hot path.  Intervals in z:
//   [2^-10, 4): 32 per octave, [2^m (1 + j/32), 2^m (1 + (j+1)/32)] -- every interval lies
//               at least 64 half-widths from the z = 0 singularity, so Y0 is tabulated
//               directly;
//   [4, 64):    uniform width 1/32 (the oscillation scale is 2 pi).
// Degree 7 on these intervals keeps every function within 2e-15 of max(1, |f|) (checked
// on the host against long-double references), with fewer Horner steps per point than a
// coarser table of higher degree.
// On each interval four functions are degree-(BTAB_NC-1) polynomials in
// t = (u - u_mid)/u_half over [z_a^2, z_b^2] (widened by 1e-6 relative), fitted on the
// host (Chebyshev interpolation in long double, converted to monomials):
//   f0 = J0,  f1 = Y0,  f2 = J1/z,  f3 = Y1/z + 2/(pi z^2)   (pole removed).
// Per interval: [u_mid, 1/u_half, f0[NC], f1[NC], f2[NC], f3[NC]].  Outside [2^-10, 64)
// the series/recurrence/asymptotic routines above are used.
#define BTAB_NC 8
#define BTAB_LOG_OCT 12            // octaves 2^-10 .. 2^2
#define BTAB_LOG_EMIN (-10)
#define BTAB_OCT_LOG2 5            // 2^5 intervals per octave
#define BTAB_PEROCT (1 << BTAB_OCT_LOG2)
#define BTAB_NLOG (BTAB_PEROCT * BTAB_LOG_OCT)
#define BTAB_W 0.03125
#define BTAB_ZLIN 4.0
#define BTAB_ZMAX 64.0
#define BTAB_NINT (BTAB_NLOG + 1920)   // (ZMAX - ZLIN) / W uniform intervals
#define BTAB_STRIDE (2 + 4 * BTAB_NC)
// double-float copy for the S/N far field: per interval 4 + 4 * BTAB_NC floats,
// [u_mid (hi, lo), 1/u_half (hi, lo)], then per power j: [J0_j (hi, lo), Y0_j (hi, lo)]
#define BTAB_DF_STRIDE (4 + 4 * BTAB_NC)
// lowest degree whose Y0 coefficients the far field evaluates in FP32 (all below 2.3e-9); J0 one
// degree lower (below 1.1e-8)
#define BTAB_FP32_DEG 5

struct BesselU { double J0, Y0, J1z, Y1z; };   // J1z = J1(z)/z, Y1z = Y1(z)/z

__device__ __forceinline__ double btab_horner(const double* c, double t) {
    double r = c[BTAB_NC - 1];
#pragma unroll
    for (int j = BTAB_NC - 2; j >= 0; --j) r = fma(r, t, c[j]);
    return r;
}

template <bool WITH1>
__device__ __forceinline__ BesselU bessel_u(const double* __restrict__ tab, double u) {
    BesselU b;
    const float zf = sqrtf((float)u);
    int i;
    if (zf < (float)BTAB_ZLIN) {
        const int bits = __float_as_int(zf);
        i = (((bits >> 23) & 255) - 127 - BTAB_LOG_EMIN) * BTAB_PEROCT + ((bits >> (23 - BTAB_OCT_LOG2)) & (BTAB_PEROCT - 1));
    } else {
        i = BTAB_NLOG + (int)((zf - (float)BTAB_ZLIN) * (float)(1.0 / BTAB_W));
    }
    if (i < 0 || i >= BTAB_NINT) {
        const double z = sqrt(u);
        const Bessel01 c = bessel01<WITH1>(z);
        b.J0 = c.J0; b.Y0 = c.Y0;
        if (WITH1) { b.J1z = c.J1 / z; b.Y1z = c.Y1 / z; }
        return b;
    }
    const double* c = tab + (size_t)i * BTAB_STRIDE;
    const double t = (u - c[0]) * c[1];
    b.J0 = btab_horner(c + 2, t);
    b.Y0 = btab_horner(c + 2 + BTAB_NC, t);
    if (WITH1) {
        b.J1z = btab_horner(c + 2 + 2 * BTAB_NC, t);
        // 1/u from a single-precision seed and two Newton steps
        double ru = (double)__frcp_rn((float)u);
        ru = ru * fma(-u, ru, 2.0);
        ru = ru * fma(-u, ru, 2.0);
        b.Y1z = btab_horner(c + 2 + 3 * BTAB_NC, t) - (2.0 / BEM_PI) * ru;
    }
    return b;
}
