// Dense Galerkin assembly of S, N (Maue form) and D on a closed polygon (Sec. II), and the
// plane-wave right-hand sides.  The Hankel kernels are evaluated by the project's own
// Bessel routines (bessel.cuh); singular pairs use closed forms (FP64), separated pairs
// double-float arithmetic (dfloat.cuh).
//
// Work decomposition: a CTA owns a T x T tile of vertex pairs (i, j) in the upper
// triangle of tiles.  It first computes the 2x2 local integrals of the (T+1)^2 segment
// pairs that touch the tile into shared memory, then combines them into vertex entries
// (vertex i = segment i as its first node, segment i-1 as its second) and writes the tile
// and, for off-diagonal tiles, its mirror (S and N are complex symmetric; D's mirror
// uses the integrals with the normal on the other segment).  Stores are column-major and
// coalesced along i.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "bessel.cuh"
#include "dfloat.cuh"
#include "kernels.h"

#define GL_MAXQ 16
__constant__ double c_glx[GL_MAXQ * (GL_MAXQ + 1) / 2];
__constant__ double c_glw[GL_MAXQ * (GL_MAXQ + 1) / 2];
__device__ __forceinline__ int gl_off(int q) { return q * (q - 1) / 2; }
#define RCP_MAX 72
__constant__ double c_rcp[RCP_MAX];     // c_rcp[k] = 1/k (c_rcp[0] = 0)
// double-float constants of the right-hand-side kernel: 1/k, Taylor coefficients of
// sin and cos ((-1)^j / (2j+1)!, (-1)^j / (2j)!), pi/2
__constant__ float2 c_rcp_df[RCP_MAX];
#define SC_TERMS 11
__constant__ float2 c_sin_df[SC_TERMS];
__constant__ float2 c_cos_df[SC_TERMS];
__constant__ float2 c_pio2_df;
// the same rules as double-float pairs: node x, weights w (1 - x) and w x
__constant__ float2 c_gx_df[GL_MAXQ * (GL_MAXQ + 1) / 2];
__constant__ float2 c_gw0_df[GL_MAXQ * (GL_MAXQ + 1) / 2];
__constant__ float2 c_gw1_df[GL_MAXQ * (GL_MAXQ + 1) / 2];
// the q = 2 rule's combination weights 1/12, 1/24, 1/(8 sqrt 3) as double-float pairs
__constant__ float2 c_q2_df[3];

static float2 host_df(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// Gauss-Legendre nodes/weights on [0,1] for q = 1..16 by Newton's method on P_q.
cudaError_t init_gauss_tables() {
    double hx[GL_MAXQ * (GL_MAXQ + 1) / 2], hw[GL_MAXQ * (GL_MAXQ + 1) / 2];
    for (int q = 1; q <= GL_MAXQ; ++q) {
        for (int i = 0; i < q; ++i) {
            double x = cos(M_PI * (i + 0.75) / (q + 0.5));
            double dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = x;
                for (int n = 2; n <= q; ++n) {
                    double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
                    p0 = p1; p1 = p2;
                }
                double pq = (q == 1) ? x : p1;
                double pqm1 = (q == 1) ? 1.0 : p0;
                dp = q * (x * pq - pqm1) / (x * x - 1.0);
                double dx = pq / dp;
                x -= dx;
                if (fabs(dx) < 1e-17) break;
            }
            // recompute derivative at the converged node
            double p0 = 1.0, p1 = x;
            for (int n = 2; n <= q; ++n) {
                double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
                p0 = p1; p1 = p2;
            }
            double pq = (q == 1) ? x : p1, pqm1 = (q == 1) ? 1.0 : p0;
            dp = q * (x * pq - pqm1) / (x * x - 1.0);
            double w = 2.0 / ((1.0 - x * x) * dp * dp);
            int o = q * (q - 1) / 2 + (q - 1 - i);      // ascending order on [0,1]
            hx[o] = 0.5 * (x + 1.0);
            hw[o] = 0.5 * w;
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(c_glx, hx, sizeof(hx));
    if (e != cudaSuccess) return e;
    float2 fx[GL_MAXQ * (GL_MAXQ + 1) / 2], fw0[GL_MAXQ * (GL_MAXQ + 1) / 2], fw1[GL_MAXQ * (GL_MAXQ + 1) / 2];
    for (int o = 0; o < GL_MAXQ * (GL_MAXQ + 1) / 2; ++o) {
        fx[o] = host_df(hx[o]);
        fw0[o] = host_df(hw[o] * (1.0 - hx[o]));
        fw1[o] = host_df(hw[o] * hx[o]);
    }
    if ((e = cudaMemcpyToSymbol(c_gx_df, fx, sizeof(fx))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_gw0_df, fw0, sizeof(fw0))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_gw1_df, fw1, sizeof(fw1))) != cudaSuccess) return e;
    {
        const long double q2[3] = {1.0L / 12.0L, 1.0L / 24.0L, 1.0L / (8.0L * sqrtl(3.0L))};
        float2 f[3];
        for (int i = 0; i < 3; ++i) {
            const float hi = (float)q2[i];
            f[i] = make_float2(hi, (float)(q2[i] - (long double)hi));
        }
        if ((e = cudaMemcpyToSymbol(c_q2_df, f, sizeof(f))) != cudaSuccess) return e;
    }
    double rc[RCP_MAX];
    rc[0] = 0.0;
    for (int k = 1; k < RCP_MAX; ++k) rc[k] = 1.0 / k;
    e = cudaMemcpyToSymbol(c_rcp, rc, sizeof(rc));
    if (e != cudaSuccess) return e;
    {
        float2 rdf[RCP_MAX], sdf[SC_TERMS], cdf[SC_TERMS];
        for (int k = 0; k < RCP_MAX; ++k) {
            const long double v = (k == 0) ? 0.0L : 1.0L / k;
            const float hi = (float)v;
            rdf[k] = make_float2(hi, (float)(v - (long double)hi));
        }
        long double fs = 1.0L, fc = 1.0L;             // (2j+1)!, (2j)!
        for (int j = 0; j < SC_TERMS; ++j) {
            if (j > 0) { fc *= (2.0L * j - 1) * (2.0L * j); fs *= (2.0L * j) * (2.0L * j + 1); }
            const long double vs = ((j & 1) ? -1.0L : 1.0L) / fs, vc = ((j & 1) ? -1.0L : 1.0L) / fc;
            const float hs = (float)vs, hc = (float)vc;
            sdf[j] = make_float2(hs, (float)(vs - (long double)hs));
            cdf[j] = make_float2(hc, (float)(vc - (long double)hc));
        }
        const long double pio2 = 1.5707963267948966192313216916397514L;
        const float hp = (float)pio2;
        const float2 pdf = make_float2(hp, (float)(pio2 - (long double)hp));
        if ((e = cudaMemcpyToSymbol(c_rcp_df, rdf, sizeof(rdf))) != cudaSuccess) return e;
        if ((e = cudaMemcpyToSymbol(c_sin_df, sdf, sizeof(sdf))) != cudaSuccess) return e;
        if ((e = cudaMemcpyToSymbol(c_cos_df, cdf, sizeof(cdf))) != cudaSuccess) return e;
        if ((e = cudaMemcpyToSymbol(c_pio2_df, &pdf, sizeof(pdf))) != cudaSuccess) return e;
    }
    return cudaMemcpyToSymbol(c_glw, hw, sizeof(hw));
}

// Coefficients of the small-r expansions (DLMF 10.8.1, 10.8.2), H_m harmonic numbers:
//   alpha_m = (-1)^m (k/2)^{2m} / (m!)^2
//   A_m = alpha_m [ i/4 - (ln(k/2) + gamma)/(2 pi) + H_m/(2 pi) ],  B_m = -alpha_m / (2 pi)
//   delta_m = (-1)^m (k/2)^{2m} / (m! (m+1)!)
//   E_m = delta_m k^2 [ -i/8 + (ln(k/2) + gamma)/(4 pi) - (H_m + H_{m+1})/(8 pi) ],
//   F_m = delta_m k^2 / (4 pi)
void series_coefficients(double k, double rmax, SeriesCoef* sc) {
    const double lk = log(0.5 * k) + BEM_EULER_GAMMA;
    double Hm = 0.0, am = 1.0, dm = 1.0;
    int nm = 0;
    for (int m = 0; m < BEM_SERIES_MAX; ++m) {
        if (m > 0) {
            Hm += 1.0 / m;
            am *= -(0.25 * k * k) / ((double)m * m);
            dm *= -(0.25 * k * k) / ((double)m * (m + 1));
        }
        const double Hm1 = Hm + 1.0 / (m + 1);
        sc->A[m] = make_double2(am * (-lk / (2 * BEM_PI) + Hm / (2 * BEM_PI)), 0.25 * am);
        sc->B[m] = -am / (2 * BEM_PI);
        sc->E[m] = make_double2(dm * k * k * (lk / (4 * BEM_PI) - (Hm + Hm1) / (8 * BEM_PI)),
                                -0.125 * dm * k * k);
        sc->F[m] = dm * k * k / (4 * BEM_PI);
        nm = m + 1;
        // stop once the m-th term at r = rmax is negligible against the leading one
        const double r2m = pow(rmax, 2.0 * m);
        if (m > 1 && fabs(am) * r2m * (1.0 + fabs(log(rmax))) < 1e-19 &&
            fabs(dm) * k * k * r2m * (1.0 + fabs(log(rmax))) < 1e-19 * k * k)
            break;
    }
    sc->nm = nm;
}


// ---------------------------------------------------------------------------------------
// Host construction of the far-field Bessel table (bessel.cuh), in long double.
// ---------------------------------------------------------------------------------------
typedef long double ld;
static const ld LD_PI = 3.141592653589793238462643383279502884L;
static const ld LD_GAMMA = 0.577215664901532860606512090082402431L;

// J0, Y0, J1, Y1 by Miller's recurrence and Neumann's expansion (z > 4)
static void host_miller(ld z, ld* J0, ld* Y0, ld* J1, ld* Y1) {
    int nstart = 2 * (int)((z + 40 + 8 * cbrtl(z)) * 0.5L);
    ld jp1 = 0, jn = 1e-40L, norm = 0, neu0 = 0, neu1 = 0, jodd = 0;
    for (int n = nstart; n >= 1; --n) {
        if ((n & 1) == 0) {
            const int k = n >> 1;
            norm += 2 * jn;
            neu0 += ((k & 1) ? -1 : 1) * jn / k;
            jodd = jp1;
        } else {
            const int k = (n + 1) >> 1;
            neu1 += ((k & 1) ? -1 : 1) * (jn - jodd) / k;
        }
        const ld jm1 = (ld)n * (2 / z) * jn - jp1;
        jp1 = jn; jn = jm1;
        if (fabsl(jn) > 1e300L) { jn *= 1e-300L; jp1 *= 1e-300L; norm *= 1e-300L; neu0 *= 1e-300L; neu1 *= 1e-300L; jodd *= 1e-300L; }
    }
    norm += jn;
    const ld s = 1 / norm, lg = logl(0.5L * z) + LD_GAMMA;
    *J0 = jn * s; *J1 = jp1 * s;
    *Y0 = (2 / LD_PI) * lg * (*J0) - (4 / LD_PI) * neu0 * s;
    *Y1 = -(2 / LD_PI) * (*J0) / z + (2 / LD_PI) * lg * (*J1) + (2 / LD_PI) * neu1 * s;
}

// the four tabulated functions at z (see bessel.cuh): J0, Y0, J1/z, Y1/z + 2/(pi z^2)
static void host_funcs(ld z, ld f[4]) {
    if (z <= 4) {
        // ascending series: J1/z and the log-free parts without dividing by z
        const ld q = 0.25L * z * z;
        ld t = 1, uu = 1, Hm = 0, sJ0 = 1, sY0 = 0, sJ1 = 1, sY1 = 1;
        for (int m = 1; m < 80; ++m) {
            t *= -q / ((ld)m * m);
            Hm += 1.0L / m;
            sJ0 += t; sY0 += Hm * t;
            uu *= -q / ((ld)m * (m + 1));
            sJ1 += uu; sY1 += (2 * Hm + 1.0L / (m + 1)) * uu;
            if (fabsl(t) < 1e-30L && fabsl(uu) < 1e-30L) break;
        }
        const ld lg = (2 / LD_PI) * logl(0.5L * z);
        const ld J0 = sJ0, Yh0 = (2 / LD_PI) * (LD_GAMMA * sJ0 - sY0);
        const ld J1z = 0.5L * sJ1, Yh1z = (2 / LD_PI) * LD_GAMMA * J1z - sY1 / (2 * LD_PI);
        f[0] = J0; f[1] = Yh0 + lg * J0; f[2] = J1z; f[3] = Yh1z + lg * J1z;
    } else {
        ld J0, Y0, J1, Y1;
        host_miller(z, &J0, &Y0, &J1, &Y1);
        f[0] = J0; f[1] = Y0; f[2] = J1 / z; f[3] = Y1 / z + 2 / (LD_PI * z * z);
    }
}

static void build_bessel_table(std::vector<double>& tab, std::vector<float>& tabf) {
    const int n = BTAB_NC;
    tab.assign((size_t)BTAB_NINT * BTAB_STRIDE, 0.0);
    tabf.assign((size_t)BTAB_NINT * BTAB_DF_STRIDE, 0.0f);
    auto put_df = [&](size_t at, ld v) {
        const float hi = (float)v;
        tabf[at] = hi;
        tabf[at + 1] = (float)(v - (ld)hi);
    };
    std::vector<ld> tk((size_t)n * n);        // monomial coefficients of T_k
    for (int k = 0; k < n; ++k) {
        for (int j = 0; j < n; ++j) {
            ld v = 0;
            if (k == 0) v = (j == 0);
            else if (k == 1) v = (j == 1);
            else v = 2 * (j > 0 ? tk[(size_t)(k - 1) * n + j - 1] : 0) - tk[(size_t)(k - 2) * n + j];
            tk[(size_t)k * n + j] = v;
        }
    }
    for (int i = 0; i < BTAB_NINT; ++i) {
        ld za, zb;
        if (i < BTAB_NLOG) {
            const int m = BTAB_LOG_EMIN + i / BTAB_PEROCT, j = i % BTAB_PEROCT;
            za = ldexpl(1.0L + j / (ld)BTAB_PEROCT, m);
            zb = ldexpl(1.0L + (j + 1) / (ld)BTAB_PEROCT, m);
        } else {
            za = (ld)BTAB_ZLIN + (i - BTAB_NLOG) * (ld)BTAB_W;
            zb = za + (ld)BTAB_W;
        }
        za *= 1 - 1e-6L;
        zb *= 1 + 1e-6L;
        const ld ua = za * za, ub = zb * zb;
        const ld um = 0.5L * (ua + ub), uh = 0.5L * (ub - ua);
        tab[(size_t)i * BTAB_STRIDE] = (double)um;
        tab[(size_t)i * BTAB_STRIDE + 1] = (double)(1.0L / uh);
        put_df((size_t)i * BTAB_DF_STRIDE, um);
        put_df((size_t)i * BTAB_DF_STRIDE + 2, 1.0L / uh);
        std::vector<ld> fv((size_t)4 * n);
        for (int j = 0; j < n; ++j) {
            const ld tj = cosl(LD_PI * (j + 0.5L) / n);
            ld f[4];
            host_funcs(sqrtl(um + uh * tj), f);
            for (int q = 0; q < 4; ++q) fv[(size_t)q * n + j] = f[q];
        }
        for (int q = 0; q < 4; ++q) {
            std::vector<ld> a(n, 0), mono(n, 0);
            for (int k = 0; k < n; ++k) {
                ld sum = 0;
                for (int j = 0; j < n; ++j) sum += fv[(size_t)q * n + j] * cosl(LD_PI * k * (j + 0.5L) / n);
                a[k] = (k == 0 ? 1.0L : 2.0L) * sum / n;
            }
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < n; ++j) mono[j] += a[k] * tk[(size_t)k * n + j];
            for (int j = 0; j < n; ++j) tab[(size_t)i * BTAB_STRIDE + 2 + (size_t)q * n + j] = (double)mono[j];
            // the double-float copy holds the kernel's factors: J0 / 4 and -Y0 / 4, so that its
            // two polynomials give (i/4) H0 = (-Y0/4, J0/4) directly (exact power-of-two scaling)
            if (q < 2)
                for (int j = 0; j < n; ++j)
                    put_df((size_t)i * BTAB_DF_STRIDE + 4 * (j + 1) + 2 * q, (q == 0 ? 0.25L : -0.25L) * mono[j]);
        }
    }
}

// The tables depend on nothing but the fit, so the host copy is built once per process;
// each handle uploads its own device copy (from its memory provider) at its first assembly.
static std::mutex g_btab_mutex;
static std::vector<double> g_btab_host;
static std::vector<float> g_btabf_host;

static bem_status bessel_table(bem_ctx* h, const double** out, const float4** outf) {
    if (!h->btab || !h->btabf) {
        {
            std::lock_guard<std::mutex> lk(g_btab_mutex);
            if (g_btab_host.empty()) build_bessel_table(g_btab_host, g_btabf_host);
        }
        // all or nothing: the handle keeps both tables, filled, or neither (a failed
        // allocation or copy must not leave one set for the next call to use)
        const size_t nb = g_btab_host.size() * sizeof(double), nf = g_btabf_host.size() * sizeof(float);
        double* tb = nullptr;
        float4* tf = nullptr;
        cudaError_t e = bem_dmalloc(h, (void**)&tb, nb);
        if (e == cudaSuccess) e = bem_dmalloc(h, (void**)&tf, nf);
        if (e == cudaSuccess) e = cudaMemcpy(tb, g_btab_host.data(), nb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(tf, g_btabf_host.data(), nf, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            bem_dfree(h, tf);
            bem_dfree(h, tb);
            return bem_cuda_check(h, e, "Bessel tables");
        }
        bem_dfree(h, h->btabf);
        bem_dfree(h, h->btab);
        h->btab = tb;
        h->btabf = tf;
    }
    *out = h->btab;
    *outf = h->btabf;
    return BEM_OK;
}

struct AsmParams {
    int N;
    double k;
    const double* seg;   // SoA x0[N], y0[N], tx[N], ty[N], h[N]
    cplx *S, *W, *D;
    int64_t ld;
    int nT;
    const double* btab;   // far-field Bessel table
    const float4* btabf;  // its J0, Y0 part as double-float pairs
    unsigned long long* qpts;   // Gauss points of separated pairs (accumulated)
    const cplx* near;     // self / adjacent pair table (k_near_pairs)
    int* rexpS;           // if set: atomic max of the exponent fields per column of S, W
    int* rexpW;           //   (W's entries with cyclic |i - j| <= wband left out)
    int wband;
    double2* kpart;       // if set: per tile column slot s and row i, the sum over the tile's
                          //   columns of N's k^2 term (kpart[s N + i]; see k_assemble_sn)
    SeriesCoef sc;
};

struct SegV { double x0, y0, tx, ty, h; };

__device__ __forceinline__ SegV load_seg(const double* seg, int N, int e) {
    SegV s;
    s.x0 = seg[e]; s.y0 = seg[N + e]; s.tx = seg[2 * N + e]; s.ty = seg[3 * N + e]; s.h = seg[4 * N + e];
    return s;
}

// ---------------------------------------------------------------------------------------
// pair integrals: I[ab] = int_e int_f lambda_a(s) lambda_b(t) g2, J: normal on f, Jt: on e
// ---------------------------------------------------------------------------------------

// self pair, closed form: with u = |s - t| the integral reduces to
//   h^2 sum_m h^{2m} [A_m T_ab(2m) + B_m (ln h T_ab(2m) + L_ab(2m))]
// where T_ab(p) = int_0^1 u^p w_ab(u) du, L_ab(p) = int_0^1 u^p ln u w_ab(u) du and
// w_11 = w_00 = 2/3 - u + u^3/3, w_01 = w_10 = 1/3 - u^3/3.
__device__ void pair_self(double h, const SeriesCoef& sc, cplx I[4]) {
    const double lnh = log(h);
    cplx i11 = cmk(0, 0), i01 = cmk(0, 0);
    double h2m = h * h;
    for (int m = 0; m < sc.nm; ++m) {
        // 1/(p + i) from the reciprocal table (p = 2m; FP64 division is a long sequence on
        // GB300's narrow FP64 pipe)
        const double r1 = c_rcp[2 * m + 1], r2 = c_rcp[2 * m + 2], r4 = c_rcp[2 * m + 4];
        const double T11 = (2.0 / 3.0) * r1 - r2 + (1.0 / 3.0) * r4;
        const double L11 = -(2.0 / 3.0) * (r1 * r1) + r2 * r2 - (1.0 / 3.0) * (r4 * r4);
        const double T01 = (1.0 / 3.0) * r1 - (1.0 / 3.0) * r4;
        const double L01 = -(1.0 / 3.0) * (r1 * r1) + (1.0 / 3.0) * (r4 * r4);
        const cplx A = sc.A[m];
        const double B = sc.B[m];
        i11.x += h2m * (A.x * T11 + B * (lnh * T11 + L11));
        i11.y += h2m * (A.y * T11);
        i01.x += h2m * (A.x * T01 + B * (lnh * T01 + L01));
        i01.y += h2m * (A.y * T01);
        h2m *= h * h;
    }
    I[0] = i11; I[3] = i11; I[1] = i01; I[2] = i01;
}

// adjacent pair, f follows e (shared vertex P = end of e = start of f).  u = sigma/h_e
// (x = P - sigma t_e), v = tau/h_f (y = P + tau t_f); triangles v <= u and u < v in Duffy
// coordinates (rho, w), r = rho R(w).  The rho integrals are closed form, w by 16-point
// Gauss.  One call gives the contribution of one node (triangle tri, Gauss node iw): the
// 32 nodes map onto the lanes of a warp (k_near_pairs).
template <bool WD>
__device__ void adjacent_node(const SegV& e, const SegV& f, const SeriesCoef& sc, int tri, int iw, cplx I[4],
                              cplx J[4], cplx Jt[4]) {
    const int qw = 16;
    const double nfx = f.ty, nfy = -f.tx, nex = e.ty, ney = -e.tx;
    const double cef = e.tx * nfx + e.ty * nfy;        // t_e . nu_f
    const double cfe = -(f.tx * nex + f.ty * ney);     // -t_f . nu_e
    const double hh = e.h * f.h;
    const double w = c_glx[gl_off(qw) + iw], wt = c_glw[gl_off(qw) + iw] * hh;
    double Rx, Ry;
    // polynomial coefficients (c0, c1, c2) in rho of lambda_a^e lambda_b^f
    double c[4][3];
    double sfac, tfac;
    if (tri == 0) {
        Rx = e.h * e.tx + w * f.h * f.tx; Ry = e.h * e.ty + w * f.h * f.ty;
        c[0][0] = 0; c[0][1] = 1; c[0][2] = -w;            // (0,0)
        c[1][0] = 0; c[1][1] = 0; c[1][2] = w;             // (0,1)
        c[2][0] = 1; c[2][1] = -(1 + w); c[2][2] = w;      // (1,0)
        c[3][0] = 0; c[3][1] = w; c[3][2] = -w;            // (1,1)
        sfac = 1.0; tfac = w;
    } else {
        Rx = w * e.h * e.tx + f.h * f.tx; Ry = w * e.h * e.ty + f.h * f.ty;
        c[0][0] = 0; c[0][1] = w; c[0][2] = -w;
        c[1][0] = 0; c[1][1] = 0; c[1][2] = w;
        c[2][0] = 1; c[2][1] = -(1 + w); c[2][2] = w;
        c[3][0] = 0; c[3][1] = 1; c[3][2] = -w;
        sfac = w; tfac = 1.0;
    }
    const double R2 = Rx * Rx + Ry * Ry;
    const double lnR = 0.5 * log(R2);
    cplx Gj[3] = {cmk(0, 0), cmk(0, 0), cmk(0, 0)};
    cplx Hj[3] = {cmk(0, 0), cmk(0, 0), cmk(0, 0)};
    double R2m = 1.0;
    for (int m = 0; m < sc.nm; ++m) {
        for (int j = 0; j < 3; ++j) {
            // 1/a and 1/b (a = 2 + j + 2m, b = a + 1) from the reciprocal table
            const double ra = c_rcp[2 + j + 2 * m];
            Gj[j].x += R2m * ((sc.A[m].x + sc.B[m] * lnR) * ra - sc.B[m] * (ra * ra));
            Gj[j].y += R2m * (sc.A[m].y * ra);
            if (WD) {
                const double rb = c_rcp[3 + j + 2 * m];
                Hj[j].x += R2m * ((sc.E[m].x + sc.F[m] * lnR) * rb - sc.F[m] * (rb * rb));
                Hj[j].y += R2m * (sc.E[m].y * rb);
            }
        }
        R2m *= R2;
    }
    const double Hs = -1.0 / (2.0 * BEM_PI * R2);
    for (int ab = 0; ab < 4; ++ab) {
        cplx si = cmk(0, 0);
        for (int j = 0; j < 3; ++j) { si.x += c[ab][j] * Gj[j].x; si.y += c[ab][j] * Gj[j].y; }
        I[ab] = cmk(wt * si.x, wt * si.y);
        if (WD) {
            cplx sd = cmk(0, 0);
            for (int j = 0; j < 3; ++j) {
                sd.x += c[ab][j] * (Hs * c_rcp[j + 1] + Hj[j].x);
                sd.y += c[ab][j] * Hj[j].y;
            }
            const double fJ = wt * e.h * sfac * cef, fJt = wt * f.h * tfac * cfe;
            J[ab] = cmk(fJ * sd.x, fJ * sd.y);
            Jt[ab] = cmk(fJt * sd.x, fJt * sd.y);
        }
    }
}

// Self and adjacent pair integrals of every segment, one warp per segment e: lanes
// (tri, iw) evaluate the 32 Duffy nodes of the pair (e, e+1) and are summed by shuffles;
// lane 0 adds the closed-form self pair.  near[e * NEAR_STRIDE + ...]:
//   [0..3] I(e,e), [4] M0(e,e), [5..8] I(e,e+1), [9] M0(e,e+1), [10..13] J(e,e+1),
//   [14..17] Jt(e,e+1);  M0 = sum_ab I_ab / (h_e h_f) (the pair's term of N's Maue form).
#define NEAR_STRIDE 18
template <bool WD>
__global__ void __launch_bounds__(256) k_near_pairs(const double* __restrict__ seg, int N, SeriesCoef sc,
                                                    cplx* __restrict__ near) {
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= N) return;                  // whole warps leave together
    const int f = (e + 1) % N;
    const SegV se = load_seg(seg, N, e), sf = load_seg(seg, N, f);
    cplx I[4], J[4], Jt[4];
    adjacent_node<WD>(se, sf, sc, lane >> 4, lane & 15, I, J, Jt);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) {
            I[q].x += __shfl_xor_sync(0xffffffffu, I[q].x, o);
            I[q].y += __shfl_xor_sync(0xffffffffu, I[q].y, o);
            if (WD) {
                J[q].x += __shfl_xor_sync(0xffffffffu, J[q].x, o);
                J[q].y += __shfl_xor_sync(0xffffffffu, J[q].y, o);
                Jt[q].x += __shfl_xor_sync(0xffffffffu, Jt[q].x, o);
                Jt[q].y += __shfl_xor_sync(0xffffffffu, Jt[q].y, o);
            }
        }
    }
    if (lane != 0) return;
    cplx* out = near + (size_t)e * NEAR_STRIDE;
    cplx Is[4];
    pair_self(se.h, sc, Is);
    const cplx ms = cadd(cadd(Is[0], Is[1]), cadd(Is[2], Is[3]));
    const cplx ma = cadd(cadd(I[0], I[1]), cadd(I[2], I[3]));
    for (int q = 0; q < 4; ++q) {
        out[q] = Is[q];
        out[5 + q] = I[q];
        out[10 + q] = WD ? J[q] : cmk(0, 0);
        out[14 + q] = WD ? Jt[q] : cmk(0, 0);
    }
    out[4] = cscale(ms, 1.0 / (se.h * se.h));
    out[9] = cscale(ma, 1.0 / (se.h * sf.h));
}

// near-pair integrals from the table: cyc = 0 self, cyc = 1 adjacent in either order
// (f = e - 1 swaps the roles of the segments: (a,b) -> (b,a), J <-> Jt)
__device__ __forceinline__ void near_from_table(const cplx* __restrict__ near, int N, int e, int f, int cyc,
                                                cplx I[4], cplx J[4], cplx Jt[4], cplx& M0) {
    if (cyc == 0) {
        const cplx* t = near + (size_t)e * NEAR_STRIDE;
        for (int q = 0; q < 4; ++q) { I[q] = t[q]; J[q] = cmk(0, 0); Jt[q] = cmk(0, 0); }
        M0 = t[4];
    } else if (f == (e + 1) % N) {
        const cplx* t = near + (size_t)e * NEAR_STRIDE;
        for (int q = 0; q < 4; ++q) { I[q] = t[5 + q]; J[q] = t[10 + q]; Jt[q] = t[14 + q]; }
        M0 = t[9];
    } else {
        const cplx* t = near + (size_t)f * NEAR_STRIDE;
        const int sw[4] = {0, 2, 1, 3};
        for (int q = 0; q < 4; ++q) { I[q] = t[5 + sw[q]]; J[q] = t[14 + sw[q]]; Jt[q] = t[10 + sw[q]]; }
        M0 = t[9];
    }
}

// separated pair: q x q tensor Gauss-Legendre
template <bool WD>
__device__ void pair_gauss(int q, const SegV& e, const SegV& f, double k, const double* __restrict__ btab,
                           cplx I[4], cplx J[4], cplx Jt[4]) {
    const double* xs = c_glx + gl_off(q);
    const double* ws = c_glw + gl_off(q);
    const double nfx = f.ty, nfy = -f.tx, nex = e.ty, ney = -e.tx;
    cplx a00 = cmk(0, 0), a01 = cmk(0, 0), a10 = cmk(0, 0), a11 = cmk(0, 0);
    cplx d00 = cmk(0, 0), d01 = cmk(0, 0), d10 = cmk(0, 0), d11 = cmk(0, 0);
    cplx t00 = cmk(0, 0), t01 = cmk(0, 0), t10 = cmk(0, 0), t11 = cmk(0, 0);
    const double k2 = k * k, k2q = 0.25 * k2;
    // y - x = (f.x0 - e.x0) + t h_f t_f - s h_e t_e
    const double bx = f.x0 - e.x0, by = f.y0 - e.y0;
    const double ux = e.h * e.tx, uy = e.h * e.ty, vx = f.h * f.tx, vy = f.h * f.ty;
    for (int i = 0; i < q; ++i) {
        const double s = xs[i];
        const double ws0 = ws[i] * (1.0 - s), ws1 = ws[i] * s;
        const double cx = bx - s * ux, cy = by - s * uy;
        for (int j = 0; j < q; ++j) {
            const double t = xs[j];
            const double wt0 = ws[j] * (1.0 - t), wt1 = ws[j] * t;
            const double dx = fma(t, vx, cx), dy = fma(t, vy, cy);
            const double r2 = fma(dx, dx, dy * dy);
            const BesselU b = bessel_u<WD>(btab, k2 * r2);
            const double gr = -0.25 * b.Y0, gi = 0.25 * b.J0;
            const double w00 = ws0 * wt0, w01 = ws0 * wt1, w10 = ws1 * wt0, w11 = ws1 * wt1;
            a00.x = fma(w00, gr, a00.x); a00.y = fma(w00, gi, a00.y);
            a01.x = fma(w01, gr, a01.x); a01.y = fma(w01, gi, a01.y);
            a10.x = fma(w10, gr, a10.x); a10.y = fma(w10, gi, a10.y);
            a11.x = fma(w11, gr, a11.x); a11.y = fma(w11, gi, a11.y);
            if (WD) {
                // -(i k/4) H1(k r) / r = (k^2/4) (Y1/z - i J1/z)
                const double fr = k2q * b.Y1z, fi = -k2q * b.J1z;
                const double dnf = dx * nfx + dy * nfy, dne = -(dx * nex + dy * ney);
                d00.x += w00 * dnf * fr; d00.y += w00 * dnf * fi;
                d01.x += w01 * dnf * fr; d01.y += w01 * dnf * fi;
                d10.x += w10 * dnf * fr; d10.y += w10 * dnf * fi;
                d11.x += w11 * dnf * fr; d11.y += w11 * dnf * fi;
                t00.x += w00 * dne * fr; t00.y += w00 * dne * fi;
                t01.x += w01 * dne * fr; t01.y += w01 * dne * fi;
                t10.x += w10 * dne * fr; t10.y += w10 * dne * fi;
                t11.x += w11 * dne * fr; t11.y += w11 * dne * fi;
            }
        }
    }
    const double hh = e.h * f.h;
    I[0] = cscale(a00, hh); I[1] = cscale(a01, hh); I[2] = cscale(a10, hh); I[3] = cscale(a11, hh);
    if (WD) {
        J[0] = cscale(d00, hh); J[1] = cscale(d01, hh); J[2] = cscale(d10, hh); J[3] = cscale(d11, hh);
        Jt[0] = cscale(t00, hh); Jt[1] = cscale(t01, hh); Jt[2] = cscale(t10, hh); Jt[3] = cscale(t11, hh);
    }
}

// Gauss order for a separated pair: Bernstein-ellipse bound rho^{-2q} exp(k Im r) <= 1e-14
// with rho = a + sqrt(a^2 - 1), a = 1 + 2 gap/h (log singularity at the gap beyond the end
// of the segment) and Im r up to about gap + h on that ellipse (the Hankel kernel grows
// like exp(k Im r) off the real axis).  1e-14 of a pair's own integral keeps every entry
// within 1e-13 of the largest (self-pair) entries.  Only a threshold, so single precision
// suffices.
__device__ __forceinline__ int q_for_gap(float ratio, float kgap) {
    const float a = 1.0f + 2.0f * fmaxf(ratio, 1e-3f);
    const float rho = a + sqrtf(a * a - 1.0f);
    const int q = (int)ceilf((32.24f + kgap) / (2.0f * __logf(rho)) + 1e-3f);
    return min(16, max(2, q));
}

// single MUFU square root (relative error about 2^-22): for the threshold decisions of the
// double-float kernel (Gauss order, table interval), where only the choice depends on it
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// q_for_gap with approximate square root and division: the same bound, evaluated to about
// 2^-20, so only pairs whose bound lands within that of an integer can change order
__device__ __forceinline__ int q_for_gap_fast(float ratio, float kgap) {
    const float a = 1.0f + 2.0f * fmaxf(ratio, 1e-3f);
    const float rho = a + sqrt_approx(a * a - 1.0f);
    const int q = (int)ceilf(__fdividef(32.24f + kgap, 2.0f * __logf(rho)) + 1e-3f);
    return min(16, max(2, q));
}

template <bool WD>
__device__ void pair_moments(int e, int f, const SegV& se, const SegV& sf, const AsmParams& p,
                             cplx I[4], cplx J[4], cplx Jt[4], unsigned& npts) {
    const int N = p.N;
    int d = e - f; if (d < 0) d = -d;
    const int cyc = min(d, N - d);
    if (cyc <= 1) {
        cplx M0;
        near_from_table(p.near, N, e, f, cyc, I, J, Jt, M0);
    } else {
        const float mx = (float)(se.x0 - sf.x0) + 0.5f * (float)(se.h * se.tx - sf.h * sf.tx);
        const float my = (float)(se.y0 - sf.y0) + 0.5f * (float)(se.h * se.ty - sf.h * sf.ty);
        const float hmax = (float)fmax(se.h, sf.h);
        const float gap = fmaxf(sqrtf(mx * mx + my * my) - 0.5f * (float)(se.h + sf.h), 0.0f);
        const int q = q_for_gap(gap / hmax, (float)p.k * (gap + hmax));
        npts += (unsigned)(q * q);
        pair_gauss<WD>(q, se, sf, p.k, p.btab, I, J, Jt);
    }
}

// Tiles of the upper triangle, ordered by distance from the diagonal (the expensive tiles,
// which hold the singular and near pairs, start first): linear index L -> (ti, tj).
__device__ __forceinline__ void tile_of(int L, int nT, int& ti, int& tj) {
    // start(d) = d nT - d (d - 1)/2 tiles precede diagonal d
    int lo = 0, hi = nT - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long st = (long long)mid * nT - (long long)mid * (mid - 1) / 2;
        if (st <= L) lo = mid; else hi = mid - 1;
    }
    const int d = lo;
    ti = L - (int)((long long)d * nT - (long long)d * (d - 1) / 2);
    tj = ti + d;
}

// table interval of u = z^2 (BTAB_NINT or beyond, or negative, outside the table)
__device__ __forceinline__ int btab_index(float uhi) {
    // an interval chosen one off at its edge is evaluated at |t| within 2^-17 of 1
    const float zf = sqrt_approx(uhi);
    if (zf < (float)BTAB_ZLIN) {
        const int bits = __float_as_int(zf);
        return (((bits >> 23) & 255) - 127 - BTAB_LOG_EMIN) * BTAB_PEROCT + ((bits >> (23 - BTAB_OCT_LOG2)) & (BTAB_PEROCT - 1));
    }
    return BTAB_NLOG + (int)fminf((zf - (float)BTAB_ZLIN) * (float)(1.0 / BTAB_W), (float)BTAB_NINT);
}

// One step p <- p t + c of a compensated Horner scheme (Graillat, Langlois and Louvet,
// Algorithms for accurate, validated and fast polynomial evaluation, 2009): p is the FP32
// Horner value and e the Horner value, in FP32, of the polynomial of its rounding errors.
// The product p t.hi splits exactly into prod + pe (FMA) and prod + c.hi into s + sg
// (two-sum); the error polynomial takes e t + pe + sg plus the parts the FP32 value leaves
// out, p t.lo and c.lo (t and c double-float).  p + e then equals the double-float Horner
// value to about the same accuracy, in 12 operations per step instead of 15.
__device__ __forceinline__ void horner_comp_step(float& p, float& e, dfl t, dfl c) {
    const float prod = __fmul_rn(p, t.hi);
    const float pe = fmaf(p, t.hi, -prod);
    const float s = __fadd_rn(prod, c.hi);
    const float bb = __fsub_rn(s, prod);
    const float sg = __fadd_rn(__fsub_rn(prod, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
    e = fmaf(e, t.hi, fmaf(p, t.lo, __fadd_rn(__fadd_rn(pe, sg), c.lo)));
    p = s;
}

// (i/4) H0(z) = (-Y0(z)/4, J0(z)/4) at u = z^2 from the double-float table, which holds
// J0/4 and -Y0/4 (FP64 routines outside it)
__device__ __forceinline__ cdfl hankel_u_df(const float4* __restrict__ tab, dfl u) {
    const int i = btab_index(u.hi);
    if (i < 0 || i >= BTAB_NINT) {
        const Bessel01 b = bessel01<false>(sqrt(dfl_to(u)));
        return {dfl_from(-0.25 * b.Y0), dfl_from(0.25 * b.J0)};
    }
    const float4* c = tab + (size_t)i * (BTAB_DF_STRIDE / 4);
    const float4 h = __ldg(c);
    const dfl t = dfl_mul(dfl_sub(u, dfl{h.x, h.y}), dfl{h.z, h.w});
    // the highest degrees in FP32: Y0's coefficients of degree >= 5 are below 2.3e-9 and
    // J0's of degree >= 4 below 1.1e-8 on every interval (|t| <= 1; a quarter of that in the
    // table), so FP32 rounding there stays below 7e-16 of the result; the lower degrees in
    // double-float
    float4 cc = __ldg(c + BTAB_NC);
    float pJ = cc.x, pY = cc.z;
#pragma unroll
    for (int j = BTAB_NC - 2; j >= BTAB_FP32_DEG; --j) {
        cc = __ldg(c + 1 + j);
        pJ = fmaf(pJ, t.hi, cc.x);
        pY = fmaf(pY, t.hi, cc.z);
    }
    cc = __ldg(c + BTAB_FP32_DEG);                       // degree BTAB_FP32_DEG - 1
    pJ = fmaf(pJ, t.hi, cc.x);
    float eJ = 0.f, eY = 0.f;
    horner_comp_step(pY, eY, t, dfl{cc.z, cc.w});
#pragma unroll
    for (int j = BTAB_FP32_DEG - 2; j >= 0; --j) {
        cc = __ldg(c + 1 + j);
        horner_comp_step(pJ, eJ, t, dfl{cc.x, cc.y});
        horner_comp_step(pY, eY, t, dfl{cc.z, cc.w});
    }
    return {dfl_qts(pY, eY), dfl_qts(pJ, eJ)};
}

// Separated pair (S/N only), q x q tensor Gauss-Legendre in double-float.  b = k (y_f(0) -
// x_e(0)), ue = k h_e t_e, vf = k h_f t_f (lengths in units of 1/k, so |b + t vf - s ue|^2 is
// the Bessel argument u = (k r)^2); returns A_ab with I_ab = h_e h_f A_ab.  The sum over
// the f-nodes runs first (two row sums R_b), then the e-node weights multiply them.  Every
// sum starts from its first product (dfl_mul, the same bits as dfl_fma onto zero).
__device__ __forceinline__ void gauss_point_df(int o, int j, dfl cx, dfl cy, dfl vfx, dfl vfy,
                                               const float4* __restrict__ tab, bool first, cdfl& R0, cdfl& R1) {
    const dfl t = dfl_mk(c_gx_df[o + j]);
    const dfl dx = dfl_fma(t, vfx, cx), dy = dfl_fma(t, vfy, cy);
    const dfl u = dfl_fma(dx, dx, dfl_mul(dy, dy));   // (k r)^2: the geometry is scaled by k
    const cdfl g = hankel_u_df(tab, u);                  // (i/4) (J0 + i Y0)
    const dfl w0 = dfl_mk(c_gw0_df[o + j]), w1 = dfl_mk(c_gw1_df[o + j]);
    if (first) {
        R0 = {dfl_mul(w0, g.re), dfl_mul(w0, g.im)};
        R1 = {dfl_mul(w1, g.re), dfl_mul(w1, g.im)};
    } else {
        R0 = cdfl_fma_real(w0, g, R0);
        R1 = cdfl_fma_real(w1, g, R1);
    }
}
__device__ __forceinline__ void gauss_row_df(int o, int i, const cdfl& R0, const cdfl& R1, bool first, cdfl A[4]) {
    const dfl w0 = dfl_mk(c_gw0_df[o + i]), w1 = dfl_mk(c_gw1_df[o + i]);
    if (first) {
        A[0] = {dfl_mul(w0, R0.re), dfl_mul(w0, R0.im)};
        A[1] = {dfl_mul(w0, R1.re), dfl_mul(w0, R1.im)};
        A[2] = {dfl_mul(w1, R0.re), dfl_mul(w1, R0.im)};
        A[3] = {dfl_mul(w1, R1.re), dfl_mul(w1, R1.im)};
    } else {
        A[0] = cdfl_fma_real(w0, R0, A[0]);
        A[1] = cdfl_fma_real(w0, R1, A[1]);
        A[2] = cdfl_fma_real(w1, R0, A[2]);
        A[3] = cdfl_fma_real(w1, R1, A[3]);
    }
}
// q = 2, the far-field bulk: the four kernel values g_ij (node i on e, j on f) combine with
// the weights W_0 = (a, b), W_1 = (b, a), a = (1 + 1/sqrt 3)/4, b = (1 - 1/sqrt 3)/4, as
//   A_00 = X + Y, A_11 = X - Y, A_01 = Z + V, A_10 = Z - V,
//   X = s/12 + p/24 = (2 s + p)/24, Z = s/24 + p/12 = (s + 2 p)/24, Y = d/(8 sqrt 3), V = q/(8 sqrt 3),
// s = g11 + g22, d = g11 - g22, p = g12 + g21, q = g12 - g21 (a^2 + b^2 = 1/6, ab = 1/24,
// a^2 - b^2 = 1/(4 sqrt 3)); and M0 = sum_ab A_ab = (s + p)/4.  Returns the integrals
// I_ab = h_e h_f A_ab, the pair's hh = h_e h_f folded into the weights 1/24 and 1/(8 sqrt 3).
__device__ __forceinline__ void pair_gauss_df_2(dfl bx, dfl by, dfl uex, dfl uey, dfl vfx, dfl vfy,
                                                const float4* __restrict__ tab, dfl hh, cdfl I[4], cdfl& M0) {
    cdfl g[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const dfl sn = dfl_mk(c_gx_df[1 + i]);
        const dfl cx = dfl_sub(bx, dfl_mul(sn, uex)), cy = dfl_sub(by, dfl_mul(sn, uey));
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const dfl t = dfl_mk(c_gx_df[1 + j]);
            const dfl dx = dfl_fma(t, vfx, cx), dy = dfl_fma(t, vfy, cy);
            g[i][j] = hankel_u_df(tab, dfl_fma(dx, dx, dfl_mul(dy, dy)));
        }
    }
    const cdfl sm = cdfl_add(g[0][0], g[1][1]), df = cdfl_sub(g[0][0], g[1][1]);
    const cdfl pp = cdfl_add(g[0][1], g[1][0]), qq = cdfl_sub(g[0][1], g[1][0]);
    const dfl w24 = dfl_mul(hh, dfl_mk(c_q2_df[1])), w83 = dfl_mul(hh, dfl_mk(c_q2_df[2]));
    const cdfl sm2 = {dfl_scale(sm.re, 2.f), dfl_scale(sm.im, 2.f)}, pp2 = {dfl_scale(pp.re, 2.f), dfl_scale(pp.im, 2.f)};
    const cdfl X = cdfl_scale(w24, cdfl_add(sm2, pp)), Z = cdfl_scale(w24, cdfl_add(sm, pp2));
    const cdfl Y = cdfl_scale(w83, df), V = cdfl_scale(w83, qq);
    I[0] = cdfl_add(X, Y);
    I[3] = cdfl_sub(X, Y);
    I[1] = cdfl_add(Z, V);
    I[2] = cdfl_sub(Z, V);
    const cdfl t = cdfl_add(sm, pp);
    M0 = {dfl_scale(t.re, 0.25f), dfl_scale(t.im, 0.25f)};
}

__device__ void pair_gauss_df(int q, dfl bx, dfl by, dfl uex, dfl uey, dfl vfx, dfl vfy,
                              const float4* __restrict__ tab, cdfl A[4]) {
    const int o = gl_off(q);
    for (int i = 0; i < q; ++i) {
        const dfl s = dfl_mk(c_gx_df[o + i]);
        const dfl cx = dfl_sub(bx, dfl_mul(s, uex)), cy = dfl_sub(by, dfl_mul(s, uey));
        cdfl R0, R1;
        gauss_point_df(o, 0, cx, cy, vfx, vfy, tab, true, R0, R1);
        for (int j = 1; j < q; ++j) gauss_point_df(o, j, cx, cy, vfx, vfy, tab, false, R0, R1);
        gauss_row_df(o, i, R0, R1, i == 0, A);
    }
}

__device__ __forceinline__ int exp_field_of(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// S and N tiles with double-float far pairs.  Same decomposition as k_assemble below: one
// CTA per T x T vertex tile of the upper triangle, (T+1)^2 segment pairs staged in shared
// memory, entries combined and written with their mirror.  Segment positions are kept as
// offsets from the tile's first segment on each side, plus one tile offset, so nearby
// pairs keep their relative geometry to double-float precision.  Self and adjacent pairs
// come from the FP64 table of k_near_pairs.
template <int T>
__device__ __forceinline__ void assemble_sn_tile(const AsmParams& p, int L) {
    int ti, tj;
    tile_of(L, p.nT, ti, tj);
    constexpr int TP = T + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // pair arrays by row el and column fl, rows RS = TP + 1 apart: the entries read them with
    // one row per lane, and the padded stride puts consecutive rows in different banks
    constexpr int RS = TP + 1, PL = TP * RS;
    float4* sI = reinterpret_cast<float4*>(smem_raw);               // 4 planes [ab][el][fl], complex df
    float4* sM = sI + 4 * PL;                                        // [el][fl]: sum_ab I / (h_e h_f)
    float2* sND = reinterpret_cast<float2*>(sM + PL);               // [el][fl]: k^2 nu_e . nu_f
    // e side: 7*TP (ox, oy, ux, uy, k tx, k ty, h); f side: 9*TP (the same, then ox, oy for
    // the tile's second e-anchor)
    float2* gE = sND + PL;
    float2* gF = gE + 7 * TP;
    __shared__ int s_mexp;                                           // largest exponent field of the means
    __shared__ unsigned char eSel[TP];                               // e-anchor of each e-segment (0, 1)
    if (threadIdx.x == 0) s_mexp = 0;
    const int N = p.N;
    const int i0 = ti * T, j0 = tj * T;
    // Positions, segment vectors and tangents are kept multiplied by k, so (k r)^2 and
    // k^2 t_e . t_f come out directly.  Positions are offsets from the segment's anchor (the
    // first segment of its block of 32), and a pair's separation is (anchor difference +
    // f offset) - e offset: the same operations on the same operands whichever tile holds
    // the pair, so a segment pair on a tile boundary gets the same integrals in both tiles
    // (N's second differences then telescope exactly), while nearby pairs keep their relative
    // geometry to double-float precision.  A tile's 32 segments span at most two anchors
    // per side; the f offsets are stored with each e-anchor's difference already added.
    const double kk = p.k;
    const int aE0 = ((i0 - 1 + N) % N) & ~31;                     // e-segments in use: anchors aE0, aE1
    const int aE1 = (aE0 + 32 < N) ? aE0 + 32 : 0;
    for (int t = threadIdx.x; t < 2 * TP; t += blockDim.x) {
        const bool isE = t < TP;
        const int l = isE ? t : t - TP;
        const int s = ((isE ? i0 : j0) - 1 + l + N) % N;
        const int a_s = s & ~31;
        const SegV a = load_seg(p.seg, N, s);
        const double ax = p.seg[a_s], ay = p.seg[N + a_s];
        float2* g = isE ? gE : gF;
        const double vals[7] = {kk * (a.x0 - ax), kk * (a.y0 - ay), kk * a.h * a.tx, kk * a.h * a.ty, kk * a.tx,
                                kk * a.ty, a.h};
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const dfl v = dfl_from(vals[c]);
            g[c * TP + l] = make_float2(v.hi, v.lo);
        }
        if (isE) {
            eSel[l] = (a_s == aE0) ? 0 : 1;
        } else {
            // f offset + (anchor of f - e-anchor), for both e-anchors of the tile
            const dfl ox = dfl_mk(g[l]), oy = dfl_mk(g[TP + l]);
#pragma unroll
            for (int ae = 0; ae < 2; ++ae) {
                const int aEs = ae ? aE1 : aE0;
                const dfl adx = dfl_from(kk * (ax - p.seg[aEs])), ady = dfl_from(kk * (ay - p.seg[N + aEs]));
                const dfl bx = dfl_add(adx, ox), by = dfl_add(ady, oy);
                g[(ae ? 7 : 0) * TP + l] = make_float2(bx.hi, bx.lo);
                g[(ae ? 8 : 1) * TP + l] = make_float2(by.hi, by.lo);
            }
        }
    }
    __syncthreads();
    unsigned npts = 0;
    int mexp = 0;
    for (int pi = threadIdx.x; pi < TP * TP; pi += blockDim.x) {
        const int el = pi / TP, fl = pi % TP;
        const int er = i0 - 1 + el, fr = j0 - 1 + fl;     // in [-1, N): -1 is segment N - 1
        if (er >= N || fr >= N) continue;
        int d = er - fr; if (d < 0) d = -d;               // |d| <= N, so the cyclic distance is
        const int cyc = min(d, N - d);                    // min(|d|, N - |d|) without a modulo
        const dfl etx = dfl_mk(gE[4 * TP + el]), ety = dfl_mk(gE[5 * TP + el]);
        const dfl ftx = dfl_mk(gF[4 * TP + fl]), fty = dfl_mk(gF[5 * TP + fl]);
        const dfl nd = dfl_fma(etx, ftx, dfl_mul(ety, fty));   // k^2 nu_e . nu_f = k^2 t_e . t_f
        cdfl I[4], M0;
        if (cyc <= 1) {
            const int e = er < 0 ? er + N : er, f = fr < 0 ? fr + N : fr;
            cplx Id[4], Jd[4], Jtd[4], m;
            near_from_table(p.near, N, e, f, cyc, Id, Jd, Jtd, m);
            for (int c = 0; c < 4; ++c) I[c] = cdfl_from(Id[c]);
            M0 = cdfl_from(m);
        } else {
            // Every unordered segment pair is integrated in one orientation, the lower segment
            // index on the x side, so that its integrals have the same bits wherever they
            // are used (the pairs of a diagonal tile below its diagonal, and those of the
            // wrapped segment N - 1, are the swapped ones); then y_x'(0) - x_e'(0) =
            // (anchor difference + y-side offset) - x-side offset.
            const int e = er < 0 ? er + N : er, f = fr < 0 ? fr + N : fr;
            const bool sw = e > f;
            dfl bx, by, uex, uey, vfx, vfy, hx, hy;
            if (!sw) {
                const int fo = eSel[el] ? 7 * TP : 0;
                bx = dfl_sub(dfl_mk(gF[fo + fl]), dfl_mk(gE[el]));
                by = dfl_sub(dfl_mk(gF[fo + TP + fl]), dfl_mk(gE[TP + el]));
                uex = dfl_mk(gE[2 * TP + el]); uey = dfl_mk(gE[3 * TP + el]);
                vfx = dfl_mk(gF[2 * TP + fl]); vfy = dfl_mk(gF[3 * TP + fl]);
                hx = dfl_mk(gE[6 * TP + el]); hy = dfl_mk(gF[6 * TP + fl]);
            } else {
                // x side: segment f (offset from its anchor recomputed: the staged one holds
                // the tile's anchor difference); y side: segment e
                const int af = f & ~31, ae = e & ~31;
                const dfl adx = dfl_from(kk * (p.seg[ae] - p.seg[af])), ady = dfl_from(kk * (p.seg[N + ae] - p.seg[N + af]));
                const dfl ofx = dfl_from(kk * (p.seg[f] - p.seg[af])), ofy = dfl_from(kk * (p.seg[N + f] - p.seg[N + af]));
                bx = dfl_sub(dfl_add(adx, dfl_mk(gE[el])), ofx);
                by = dfl_sub(dfl_add(ady, dfl_mk(gE[TP + el])), ofy);
                uex = dfl_mk(gF[2 * TP + fl]); uey = dfl_mk(gF[3 * TP + fl]);
                vfx = dfl_mk(gE[2 * TP + el]); vfy = dfl_mk(gE[3 * TP + el]);
                hx = dfl_mk(gF[6 * TP + fl]); hy = dfl_mk(gE[6 * TP + el]);
            }
            // (scaled by k: kgap = k (gap + h_max) directly)
            const float kf = (float)p.k;
            const float he = kf * hx.hi, hf = kf * hy.hi;
            const float mx = bx.hi + 0.5f * (vfx.hi - uex.hi), my = by.hi + 0.5f * (vfy.hi - uey.hi);
            const float hmax = fmaxf(he, hf);
            const float gap = fmaxf(sqrt_approx(mx * mx + my * my) - 0.5f * (he + hf), 0.0f);
            const int q = q_for_gap_fast(__fdividef(gap, hmax), gap + hmax);
            npts += (unsigned)(q * q);
            const dfl hh = dfl_mul(hx, hy);
            if (q == 2) {
                pair_gauss_df_2(bx, by, uex, uey, vfx, vfy, p.btabf, hh, I, M0);   // the far-field bulk
            } else {
                cdfl A[4];
                pair_gauss_df(q, bx, by, uex, uey, vfx, vfy, p.btabf, A);
                M0 = cdfl_add(cdfl_add(A[0], A[1]), cdfl_add(A[2], A[3]));
                for (int c = 0; c < 4; ++c) I[c] = {dfl_mul(hh, A[c].re), dfl_mul(hh, A[c].im)};
            }
            if (sw) { const cdfl t = I[1]; I[1] = I[2]; I[2] = t; }   // I_ab(e, f) = I_ba(f, e)
        }
        const int ps = el * RS + fl;
        for (int c = 0; c < 4; ++c) sI[c * PL + ps] = cdfl_pack(I[c]);
        sM[ps] = cdfl_pack(M0);
        sND[ps] = make_float2(nd.hi, nd.lo);
        mexp = max(mexp, max((__float_as_int(M0.re.hi) >> 23) & 255, (__float_as_int(M0.im.hi) >> 23) & 255));
    }
    for (int o = 16; o > 0; o >>= 1) npts += __shfl_xor_sync(0xffffffffu, npts, o);
    if ((threadIdx.x & 31) == 0 && npts) atomicAdd(p.qpts, (unsigned long long)npts);
    // N's derivative term is the second difference of the segment-pair means M0 (Maue's
    // form): at low k its row sums are O(k^2) of the means, so the differences are taken
    // exactly, in fixed point with one scale per tile (|M0| 2^msh < 2^59, leaving room for
    // the k^2 term, at most 4 |M0| with k h <= 2), and every entry of N is rounded once, to
    // FP64, from that exact sum; each mean is rounded once too, which perturbs the means,
    // not the null space of the differences
    mexp = (int)__reduce_max_sync(0xffffffffu, (unsigned)mexp);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_mexp, mexp);
    __syncthreads();
    const int msh = 185 - s_mexp;
    longlong2* sMx = reinterpret_cast<longlong2*>(sM);    // the means in fixed point, in place
    if (p.W) {
        for (int pi = threadIdx.x; pi < TP * TP; pi += blockDim.x) {
            const int el = pi / TP, fl = pi % TP;
            if (i0 - 1 + el >= N || j0 - 1 + fl >= N) continue;
            const cdfl m = cdfl_unpack(sM[el * RS + fl]);
            sMx[el * RS + fl] = make_longlong2(dfl_to_fixed(m.re, msh), dfl_to_fixed(m.im, msh));
        }
    }
    const bool mirror = (ti != tj);
    // entry (i0 + il, j0 + jl) of S and N, written at (i, j)
    auto entry = [&](int il, int jl, double2& ds, double2& dw, cdfl& kt) -> bool {
        const int i = i0 + il, j = j0 + jl;
        if (i >= N || j >= N) return false;
        cdfl sv, wv = cdfl_zero();
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int el = il + 1 - a;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int fl = jl + 1 - b;
                const int ps = el * RS + fl;
                const cdfl Iab = cdfl_unpack(sI[(a * 2 + b) * PL + ps]);
                sv = (a | b) ? cdfl_add(sv, Iab) : Iab;
                // the k^2 term: - k^2 (nu_e . nu_f) I_ab
                if (p.W) wv = cdfl_fma_real(dfl_neg(dfl_mk(sND[ps])), Iab, wv);
            }
        }
        const int64_t off = (int64_t)i + (int64_t)j * p.ld;
        ds = cdfl_to(sv);
        dw = make_double2(0.0, 0.0);
        kt = wv;
        if (p.W) {
            // sum_ab sigma_a sigma_b M0(i-a, j-b) = (M0[i-1][j-1] - M0[i-1][j]) - (M0[i][j-1] - M0[i][j]),
            // plus the k^2 term, exactly in fixed point; one rounding to FP64
            const longlong2 m00 = sMx[il * RS + jl], m01 = sMx[il * RS + jl + 1];
            const longlong2 m10 = sMx[(il + 1) * RS + jl], m11 = sMx[(il + 1) * RS + jl + 1];
            const long long wr = ((m00.x - m01.x) - (m10.x - m11.x)) + dfl_to_fixed(wv.re, msh);
            const long long wi = ((m00.y - m01.y) - (m10.y - m11.y)) + dfl_to_fixed(wv.im, msh);
            dw = make_double2(fixed_to_double(wr, msh), fixed_to_double(wi, msh));
        }
        if (p.S) p.S[off] = ds;
        if (p.W) p.W[off] = dw;
        return true;
    };
    // Direct half: one warp per tile column, lane = row; the entries stay in registers for
    // the mirror.  When asked, the largest exponent fields of the written entries are
    // gathered per column (a warp reduction) and, for the mirror, per row (the slices of the
    // split products are scaled per column of S and N; N's band is left out).
    const bool track = p.rexpS != nullptr;
    __shared__ int eRow[2][32];
    float4* sK = reinterpret_cast<float4*>(gF + 9 * TP);  // T*T: the entries' k^2 terms [jl T + il]
    if (threadIdx.x < 64) eRow[threadIdx.x >> 5][threadIdx.x & 31] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NQ = (T + 7) / 8;                      // columns per warp (8 warps)
    double2 keepS[NQ], keepW[NQ];
    {
        int rS = 0, rW = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int jl = wid + 8 * q;
            if (jl >= T) break;
            double2 ds = make_double2(0.0, 0.0), dw = make_double2(0.0, 0.0);
            cdfl kt = cdfl_zero();
            int fs = 0, fw = 0;
            const bool ok = lane < T && entry(lane, jl, ds, dw, kt);
            if (!ok) kt = cdfl_zero();
            if (ok && track) {
                int d = lane + i0 - (jl + j0); if (d < 0) d = -d;
                fs = max(exp_field_of(ds.x), exp_field_of(ds.y));
                fw = (min(d, N - d) <= p.wband) ? 0 : max(exp_field_of(dw.x), exp_field_of(dw.y));
            }
            keepS[q] = ds;
            keepW[q] = dw;
            if (p.kpart && lane < T) sK[jl * T + lane] = cdfl_pack(kt);
            if (track) {
                const int cs = (int)__reduce_max_sync(0xffffffffu, (unsigned)fs);
                const int cw = (int)__reduce_max_sync(0xffffffffu, (unsigned)fw);
                if (lane == 0 && j0 + jl < N) {
                    atomicMax(p.rexpS + j0 + jl, cs);
                    atomicMax(p.rexpW + j0 + jl, cw);
                }
                rS = max(rS, fs);
                rW = max(rW, fw);
            }
        }
        if (track && mirror) {
            atomicMax(&eRow[0][lane], rS);
            atomicMax(&eRow[1][lane], rW);
        }
    }
    __syncthreads();                                     // sI is no longer read
    // N 1 = the row sums of the k^2 term exactly (the derivative term's vanish): the tile's
    // share, summed in a fixed order, goes to the slot of its tile column (its rows) and,
    // mirrored, of its tile row (the columns' sums are the mirror's row sums)
    if (p.kpart) {
        // two stages: 4 groups of 8 columns (rows' sums) or rows (columns' sums), then the 4
        // group partials (in sND's space, free now), each in a fixed order
        float4* part = reinterpret_cast<float4*>(sND);   // [2][4][T]
        const int t = threadIdx.x;
        if (t < 4 * T || (mirror && t >= 128 && t < 128 + 4 * T)) {
            const bool col = t >= 128;
            const int u = col ? t - 128 : t, g = u / T, l = u % T;
            const int m0 = 8 * g, m1 = min(T, m0 + 8);
            cdfl acc = cdfl_zero();
            for (int m = m0; m < m1; ++m) acc = cdfl_add(acc, cdfl_unpack(col ? sK[l * T + m] : sK[m * T + l]));
            part[(col ? 4 * T : 0) + g * T + l] = cdfl_pack(acc);
        }
        __syncthreads();
        if (t < T && i0 + t < N) {
            cdfl acc = cdfl_unpack(part[t]);
            for (int g = 1; g < 4; ++g) acc = cdfl_add(acc, cdfl_unpack(part[g * T + t]));
            p.kpart[(int64_t)tj * N + i0 + t] = cdfl_to(acc);
        } else if (mirror && t >= 32 && t < 32 + T && j0 + t - 32 < N) {
            const int jl = t - 32;
            cdfl acc = cdfl_unpack(part[4 * T + jl]);
            for (int g = 1; g < 4; ++g) acc = cdfl_add(acc, cdfl_unpack(part[4 * T + g * T + jl]));
            p.kpart[(int64_t)ti * N + j0 + jl] = cdfl_to(acc);
        }
    }
    if (track && mirror && threadIdx.x < 2 * T) {
        const int m = threadIdx.x / T, l = threadIdx.x % T;
        if (i0 + l < N) atomicMax((m ? p.rexpW : p.rexpS) + i0 + l, eRow[m][l]);
    }
    // mirror half: the same entries staged through shared memory (over sI), stored transposed
    if (mirror) {
        double2* stage = reinterpret_cast<double2*>(sI);   // [(jl T + il) 2 + (0: S, 1: N)]
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int jl = wid + 8 * q;
            if (jl >= T) break;
            if (lane < T) {
                stage[(jl * T + lane) * 2] = keepS[q];
                stage[(jl * T + lane) * 2 + 1] = keepW[q];
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
            const int il = idx / T, jl = idx % T;
            const int i = i0 + il, j = j0 + jl;
            if (i >= N || j >= N) continue;
            const int64_t off = (int64_t)j + (int64_t)i * p.ld;
            if (p.S) p.S[off] = stage[(jl * T + il) * 2];
            if (p.W) p.W[off] = stage[(jl * T + il) * 2 + 1];
        }
    }
}

static_assert(sizeof(AsmParams) % 4 == 0, "AsmParams is copied to shared memory in 4-byte words");

// Shared memory of one S/N tile of edge T: (T+1)^2 segment pairs in rows of T+2 (four
// integrals, the mean, k^2 nu_e . nu_f), the staged geometry and the entries' k^2 terms.
// 110 KB at T = 31 admits two CTAs per SM, 64 KB at T = 23 three and 30 KB at T = 15 four.  The smaller tiles are
// compiled for that many CTAs (at most 85 and 64 registers per thread); T = 31 is left to
// the compiler's choice (108 registers, two CTAs).
__host__ __device__ constexpr size_t asm_sn_smem(int T) {
    return (size_t)(T + 1) * (T + 2) * (4 * sizeof(float4) + sizeof(float4) + sizeof(float2)) +
           (size_t)16 * (T + 1) * sizeof(float2) + (size_t)T * T * sizeof(float4);
}
__host__ __device__ constexpr int asm_min_blocks(int T) { return T <= 15 ? 4 : (T <= 23 ? 3 : 1); }
#define ASM_TILE_DEFAULT 31
static int asm_tile_of(const bem_ctx* h) { return h->opt.asm_tile ? h->opt.asm_tile : ASM_TILE_DEFAULT; }

// one CTA per tile of one problem
template <int T>
__global__ void __launch_bounds__(256, asm_min_blocks(T)) k_assemble_sn(AsmParams p) {
    assemble_sn_tile<T>(p, (int)blockIdx.x);
}

// Many problems in one launch: persistent CTAs take tiles from one global queue (an atomic
// counter over the problems' tiles in order, the problems sorted largest first by the caller
// and each one's tiles diagonal-first), so small problems fill the GPU behind large ones.
// first[q] is the queue position of problem q's first tile; the tiles need no waits.
template <int T>
__global__ void __launch_bounds__(256, asm_min_blocks(T)) k_assemble_sn_batch(const AsmParams* __restrict__ ps,
                                                           const long long* __restrict__ first, int nprob,
                                                           long long total, unsigned long long* queue) {
    __shared__ AsmParams sp;
    __shared__ long long s_L;
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long L = (long long)atomicAdd(queue, 1ull);
            int lo = 0, hi = nprob - 1;                  // the last problem with first[q] <= L
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (first[mid] <= L) lo = mid; else hi = mid - 1;
            }
            s_L = L;
            s_q = lo;
        }
        __syncthreads();
        const long long L = s_L;
        if (L >= total) return;
        const int q = s_q;
        for (int w = threadIdx.x; w < (int)(sizeof(AsmParams) / 4); w += blockDim.x)
            reinterpret_cast<int*>(&sp)[w] = reinterpret_cast<const int*>(ps + q)[w];
        __syncthreads();
        assemble_sn_tile<T>(sp, (int)(L - first[q]));
        __syncthreads();                                 // shared state is reused by the next tile
    }
}

template <int T, bool WD>
__global__ void __launch_bounds__(256) k_assemble(AsmParams p) {
    int ti, tj;
    tile_of((int)blockIdx.x, p.nT, ti, tj);
    constexpr int TP = T + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx* sI = reinterpret_cast<cplx*>(smem_raw);                 // TP*TP*4
    cplx* sM = sI + TP * TP * 4;                                    // TP*TP: sum_ab I / (h_e h_f)
    cplx* sJ = sM + TP * TP;                                        // (WD)
    cplx* sJt = sJ + (WD ? TP * TP * 4 : 0);
    double* sND = reinterpret_cast<double*>(sJt + (WD ? TP * TP * 4 : 0));   // TP*TP: k^2 nu_e.nu_f
    double* sgE = sND + TP * TP;                                    // 5*TP
    double* sgF = sgE + 5 * TP;
    const int N = p.N;
    const int i0 = ti * T, j0 = tj * T;
    for (int t = threadIdx.x; t < TP; t += blockDim.x) {
        const int e = (i0 - 1 + t + N) % N, f = (j0 - 1 + t + N) % N;
        const SegV a = load_seg(p.seg, N, e), b = load_seg(p.seg, N, f);
        sgE[t] = a.x0; sgE[TP + t] = a.y0; sgE[2 * TP + t] = a.tx; sgE[3 * TP + t] = a.ty; sgE[4 * TP + t] = a.h;
        sgF[t] = b.x0; sgF[TP + t] = b.y0; sgF[2 * TP + t] = b.tx; sgF[3 * TP + t] = b.ty; sgF[4 * TP + t] = b.h;
    }
    __syncthreads();
    const double k2 = p.k * p.k;
    unsigned npts = 0;
    for (int pi = threadIdx.x; pi < TP * TP; pi += blockDim.x) {
        const int el = pi / TP, fl = pi % TP;
        // skip segment pairs touching only rows/cols beyond N
        if (i0 - 1 + el >= N || j0 - 1 + fl >= N) continue;
        const int e = (i0 - 1 + el + N) % N, f = (j0 - 1 + fl + N) % N;
        SegV se = {sgE[el], sgE[TP + el], sgE[2 * TP + el], sgE[3 * TP + el], sgE[4 * TP + el]};
        SegV sf = {sgF[fl], sgF[TP + fl], sgF[2 * TP + fl], sgF[3 * TP + fl], sgF[4 * TP + fl]};
        cplx I[4], J[4], Jt[4];
        // every unordered pair in one orientation (lower segment index first), so its
        // integrals have the same bits in every tile that uses them (N's second differences
        // then telescope exactly); I_ab(e, f) = I_ba(f, e), J and Jt trade places
        const bool sw = e > f;
        if (!sw) pair_moments<WD>(e, f, se, sf, p, I, J, Jt, npts);
        else pair_moments<WD>(f, e, sf, se, p, I, J, Jt, npts);
        // per-pair terms of N's Maue form: sum_ab I / (h_e h_f) and k^2 nu_e . nu_f
        const double ihh = sw ? 1.0 / (sf.h * se.h) : 1.0 / (se.h * sf.h);
        const cplx M0 = cadd(cadd(I[0], I[1]), cadd(I[2], I[3]));
        sM[pi] = cscale(M0, ihh);
        if (sw) {
            cplx t = I[1]; I[1] = I[2]; I[2] = t;
            if (WD) {
                cplx Jn[4] = {Jt[0], Jt[2], Jt[1], Jt[3]}, Jtn[4] = {J[0], J[2], J[1], J[3]};
                for (int q = 0; q < 4; ++q) { J[q] = Jn[q]; Jt[q] = Jtn[q]; }
            }
        }
        for (int q = 0; q < 4; ++q) {
            sI[pi * 4 + q] = I[q];
            if (WD) { sJ[pi * 4 + q] = J[q]; sJt[pi * 4 + q] = Jt[q]; }
        }
        sND[pi] = k2 * (se.ty * sf.ty + se.tx * sf.tx);   // nu = (t_y, -t_x): nu_e . nu_f = t_e . t_f
    }
    for (int o = 16; o > 0; o >>= 1) npts += __shfl_xor_sync(0xffffffffu, npts, o);
    if ((threadIdx.x & 31) == 0 && npts) atomicAdd(p.qpts, (unsigned long long)npts);
    __syncthreads();
    const bool mirror = (ti != tj);
    for (int pass = 0; pass < (mirror ? 2 : 1); ++pass) {
        for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
            int il, jl;
            if (pass == 0) { il = idx % T; jl = idx / T; } else { jl = idx % T; il = idx / T; }
            const int i = i0 + il, j = j0 + jl;
            if (i >= N || j >= N) continue;
            cplx s = cmk(0, 0), w = cmk(0, 0), dd = cmk(0, 0);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int el = il + 1 - a;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int fl = jl + 1 - b;
                    const int pi = el * TP + fl;
                    const cplx Iab = sI[pi * 4 + a * 2 + b];
                    s = cadd(s, Iab);
                    if (p.W) {
                        // the k^2 term: - k^2 (nu_e . nu_f) I_ab
                        const double nd = sND[pi];
                        w.x -= nd * Iab.x;
                        w.y -= nd * Iab.y;
                    }
                    if (WD) dd = cadd(dd, (pass == 0 ? sJ : sJt)[pi * 4 + a * 2 + b]);
                }
            }
            if (p.W) {
                // the derivative term sum_ab sigma_a sigma_b M0(i-a, j-b) as the second
                // difference (M0[i-1][j-1] - M0[i-1][j]) - (M0[i][j-1] - M0[i][j]): each
                // difference of two close means is exact, so N's vanishing row sums of this
                // term are kept to the rounding of the small differences (at low k they
                // carry the O(k^2) row sums of N)
                const cplx m00 = sM[il * TP + jl], m01 = sM[il * TP + jl + 1];
                const cplx m10 = sM[(il + 1) * TP + jl], m11 = sM[(il + 1) * TP + jl + 1];
                w.x += (m00.x - m01.x) - (m10.x - m11.x);
                w.y += (m00.y - m01.y) - (m10.y - m11.y);
            }
            const int64_t off = (pass == 0) ? ((int64_t)i + (int64_t)j * p.ld) : ((int64_t)j + (int64_t)i * p.ld);
            if (p.S) p.S[off] = s;
            if (p.W) p.W[off] = w;
            if (WD && p.D) p.D[off] = dd;
        }
    }
}

// per-segment geometry (SoA) and chord statistics: stats[0] = min h, stats[1] = max h (by
// atomics on the ordered bit patterns of positive doubles); the sum of h is formed by
// k_sum_h in a fixed order, so the mean chord is the same on every run
__global__ void k_geometry(const double* verts, int N, double* seg, double* stats) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int f = (e + 1) % N;
    const double x0 = verts[2 * e], y0 = verts[2 * e + 1];
    const double dx = verts[2 * f] - x0, dy = verts[2 * f + 1] - y0;
    const double h = sqrt(dx * dx + dy * dy);
    seg[e] = x0; seg[N + e] = y0; seg[2 * N + e] = dx / h; seg[3 * N + e] = dy / h; seg[4 * N + e] = h;
    unsigned long long hb = __double_as_longlong(h);
    atomicMin(reinterpret_cast<unsigned long long*>(stats), hb);
    atomicMax(reinterpret_cast<unsigned long long*>(stats + 1), hb);
}

// stats[2] = sum of h over the N segments, one CTA, fixed summation order
__global__ void __launch_bounds__(1024) k_sum_h(const double* hseg, int N, double* stats) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int e = threadIdx.x; e < N; e += blockDim.x) s += hseg[e];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) stats[2] = part[0];
}

bem_status launch_geometry(bem_ctx* h, const double* verts, int64_t N, double* stats_dev) {
    double init[3] = {1e300, 0.0, 0.0};
    BEM_CUDA(h, cudaMemcpyAsync(stats_dev, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
    BEM_TIMED(h, "k_geometry", (k_geometry<<<(unsigned)((N + 255) / 256), 256, 0, h->stream>>>(verts, (int)N, h->seg, stats_dev)));
    BEM_LAUNCH(h, "k_geometry");
    BEM_TIMED(h, "k_sum_h", (k_sum_h<<<1, 1024, 0, h->stream>>>(h->seg + 4 * N, (int)N, stats_dev)));
    BEM_LAUNCH(h, "k_sum_h");
    return BEM_OK;
}

template <int T, bool WD>
static bem_status run_assemble(bem_ctx* h, AsmParams& p) {
    constexpr int TP = T + 1;
    const size_t smem = (size_t)TP * TP * 4 * sizeof(cplx) * (WD ? 3 : 1) + (size_t)TP * TP * (sizeof(cplx) + sizeof(double)) +
                        10 * TP * sizeof(double);
    BEM_CUDA(h, cudaFuncSetAttribute(k_assemble<T, WD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    p.nT = (p.N + T - 1) / T;
    const unsigned grid = (unsigned)((int64_t)p.nT * (p.nT + 1) / 2);
    BEM_TIMED(h, "k_assemble", (k_assemble<T, WD><<<grid, 256, smem, h->stream>>>(p)));
    BEM_LAUNCH(h, "k_assemble");
    return BEM_OK;
}

// k1[i] = sum over the tile slots s of kpart[s N + i], in slot order
__global__ void k_sum_slots(const double2* __restrict__ kpart, int nslots, int N, cplx* k1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    cplx t = cmk(0, 0);
    for (int s = 0; s < nslots; ++s) t = cadd(t, kpart[(int64_t)s * N + i]);
    k1[i] = t;
}

template <int T>
static bem_status run_assemble_sn(bem_ctx* h, AsmParams& p) {
    const size_t smem = asm_sn_smem(T);
    BEM_CUDA(h, cudaFuncSetAttribute(k_assemble_sn<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    p.nT = (p.N + T - 1) / T;
    const unsigned grid = (unsigned)((int64_t)p.nT * (p.nT + 1) / 2);
    BEM_TIMED(h, "k_assemble", (k_assemble_sn<T><<<grid, 256, smem, h->stream>>>(p)));
    BEM_LAUNCH(h, "k_assemble");
    if (p.kpart) {
        BEM_TIMED(h, "k_sum_slots", (k_sum_slots<<<(unsigned)((p.N + 255) / 256), 256, 0, h->stream>>>(p.kpart, p.nT, p.N, h->k1)));
        BEM_LAUNCH(h, "k_sum_slots");
    }
    return BEM_OK;
}

// Tables, near-pair integrals and output buffers of one assembly on h's stream; *near is a
// stream-ordered temporary the caller frees (asm_finish) after the tiles have run.
static bem_status asm_prepare(bem_ctx* h, unsigned ops, AsmParams& p, cplx** near_out, int T) {
    p.N = (int)h->N;
    p.k = h->k;
    p.seg = h->seg;
    p.S = (ops & BEM_OP_S) ? h->S : nullptr;
    p.W = (ops & BEM_OP_W) ? h->W : nullptr;
    p.D = (ops & BEM_OP_D) ? h->D : nullptr;
    p.ld = h->N;
    p.qpts = h->qpts;
    BEM_CUDA(h, cudaMemsetAsync(h->qpts, 0, sizeof(unsigned long long), h->stream));
    series_coefficients(h->k, 2.0 * (h->general ? h->hmax : h->hbar), &p.sc);
    bem_status st = bessel_table(h, &p.btab, &p.btabf);
    if (st != BEM_OK) return st;
    cplx* near = nullptr;
    BEM_CUDA(h, bem_dmalloc_async(h, (void**)&near, sizeof(cplx) * NEAR_STRIDE * (size_t)h->N));
    *near_out = near;
    const unsigned gnear = (unsigned)((h->N + 7) / 8);
    if (ops & BEM_OP_D) {
        BEM_TIMED(h, "k_near_pairs", (k_near_pairs<true><<<gnear, 256, 0, h->stream>>>(h->seg, (int)h->N, p.sc, near)));
    } else {
        BEM_TIMED(h, "k_near_pairs", (k_near_pairs<false><<<gnear, 256, 0, h->stream>>>(h->seg, (int)h->N, p.sc, near)));
    }
    BEM_LAUNCH(h, "k_near_pairs");
    p.near = near;
    p.rexpS = p.rexpW = nullptr;
    p.wband = -1;
    p.kpart = nullptr;
    h->rexp_valid = false;
    h->k1_valid = false;
    if (!(ops & BEM_OP_D)) {
        // N's row sums (exact: those of its k^2 term), per tile slot, for the filter's
        // constant-vector correction
        const int64_t nT = (h->N + T - 1) / T;
        if (!h->k1) BEM_CUDA(h, bem_dmalloc(h, (void**)&h->k1, sizeof(cplx) * (size_t)h->N));
        if (h->kpart && h->kpart_slots < nT) {
            bem_dfree(h, h->kpart);
            h->kpart = nullptr;
            h->kpart_slots = 0;
        }
        if (!h->kpart) {
            BEM_CUDA(h, bem_dmalloc(h, (void**)&h->kpart, sizeof(double2) * (size_t)nT * h->N));
            h->kpart_slots = nT;
        }
        p.kpart = h->kpart;
    }
    if (!(ops & BEM_OP_D) && h->opt.prec == BEM_MIXED_BF16) {
        if (!h->rexp) BEM_CUDA(h, bem_dmalloc(h, (void**)&h->rexp, sizeof(int) * 2 * (size_t)h->N));
        BEM_CUDA(h, cudaMemsetAsync(h->rexp, 0, sizeof(int) * 2 * (size_t)h->N, h->stream));
        p.rexpS = h->rexp;
        p.rexpW = h->rexp + h->N;
        p.wband = (int)std::min<int64_t>(TC_W_BAND, (h->N - 1) / 2);
    }
    return BEM_OK;
}

static void asm_finish(bem_ctx* h, const AsmParams& p, cplx* near, bem_status st) {
    if (st == BEM_OK && p.rexpS) h->rexp_valid = true;
    if (st == BEM_OK && p.kpart) h->k1_valid = true;
    bem_dfree_async(h, near);
}

bem_status launch_assemble(bem_ctx* h, unsigned ops) {
    AsmParams p;
    cplx* near = nullptr;
    const int T = (ops & BEM_OP_D) ? 15 : asm_tile_of(h);
    bem_status st = asm_prepare(h, ops, p, &near, T);
    if (st == BEM_OK) {
        if (ops & BEM_OP_D) st = run_assemble<15, true>(h, p);
        else if (T == 15) st = run_assemble_sn<15>(h, p);
        else if (T == 23) st = run_assemble_sn<23>(h, p);
        else st = run_assemble_sn<31>(h, p);
    }
    asm_finish(h, p, near, st);
    return st;
}

// The batched assembly with tile edge T (launch_assemble_batch below).
template <int T>
static bem_status assemble_batch_tiles(bem_ctx** hs, int nprob) {
    bem_ctx* h0 = hs[0];
    std::vector<AsmParams> ps(nprob);
    std::vector<cplx*> nears(nprob, nullptr);
    bem_status st = BEM_OK;
    for (int q = 0; q < nprob && st == BEM_OK; ++q) {
        st = asm_prepare(hs[q], BEM_OP_S | BEM_OP_W, ps[q], &nears[q], T);
        ps[q].nT = (ps[q].N + T - 1) / T;
    }
    // the largest problems' tiles first
    std::vector<int> order(nprob);
    for (int q = 0; q < nprob; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ps[a].N > ps[b].N; });
    std::vector<AsmParams> sorted(nprob);
    std::vector<long long> first(nprob);
    long long total = 0;
    for (int r = 0; r < nprob; ++r) {
        sorted[r] = ps[order[r]];
        first[r] = total;
        total += (long long)sorted[r].nT * (sorted[r].nT + 1) / 2;
    }
    AsmParams* dps = nullptr;
    long long* dfirst = nullptr;
    unsigned long long* queue = nullptr;
    std::vector<cudaEvent_t> evs;
    if (st == BEM_OK) {
        const size_t bytes = sizeof(AsmParams) * nprob + sizeof(long long) * nprob + 256;
        void* buf = nullptr;
        const cudaError_t ae = bem_dmalloc_async(h0, &buf, bytes);
        if (ae != cudaSuccess) {
            st = bem_cuda_check(h0, ae, "batch assembly parameters");
        } else {
            dps = (AsmParams*)buf;
            dfirst = (long long*)((char*)buf + sizeof(AsmParams) * nprob);
            queue = (unsigned long long*)((char*)dfirst + sizeof(long long) * nprob);
        }
    }
    if (st == BEM_OK) {
        // the other handles' preparation before the launch
        for (int q = 1; q < nprob; ++q) {
            cudaEvent_t e = bem_event_get(hs[q]);
            cudaEventRecord(e, hs[q]->stream);
            cudaStreamWaitEvent(h0->stream, e, 0);
            evs.push_back(e);
        }
        cudaMemcpyAsync(dps, sorted.data(), sizeof(AsmParams) * nprob, cudaMemcpyHostToDevice, h0->stream);
        cudaMemcpyAsync(dfirst, first.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice, h0->stream);
        cudaMemsetAsync(queue, 0, sizeof(unsigned long long), h0->stream);
        const size_t smem = asm_sn_smem(T);
        cudaError_t e = cudaFuncSetAttribute(k_assemble_sn_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per = 0, nsm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_assemble_sn_batch<T>, 256, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h0->device);
        if (e != cudaSuccess) st = bem_cuda_check(h0, e, "batch assembly launch setup");
        if (st == BEM_OK) {
            const long long ctas = std::min<long long>(total, (long long)std::max(per, 1) * nsm);
            BEM_TIMED(h0, "k_assemble_batch", (k_assemble_sn_batch<T><<<(unsigned)ctas, 256, smem, h0->stream>>>(
                                                   dps, dfirst, nprob, total, queue)));
            cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) st = bem_cuda_check(h0, le, "k_assemble_sn_batch");
        }
        // everything after the launch, per handle, waits for it
        cudaEvent_t done = bem_event_get(h0);
        cudaEventRecord(done, h0->stream);
        for (int q = 1; q < nprob; ++q) cudaStreamWaitEvent(hs[q]->stream, done, 0);
        evs.push_back(done);
        for (int q = 0; q < nprob && st == BEM_OK; ++q) {
            bem_ctx* h = hs[q];
            BEM_TIMED(h, "k_sum_slots", (k_sum_slots<<<(unsigned)((ps[q].N + 255) / 256), 256, 0, h->stream>>>(
                                             ps[q].kpart, ps[q].nT, ps[q].N, h->k1)));
            cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) st = bem_cuda_check(h, le, "k_sum_slots");
        }
        bem_dfree_async(h0, dps);
        cudaStreamSynchronize(h0->stream);         // the host-side parameter arrays
    }
    for (int q = 0; q < nprob; ++q) asm_finish(hs[q], ps[q], nears[q], st);
    for (size_t i = 0; i + 1 < evs.size(); ++i) hs[i + 1]->evpool.push_back(evs[i]);
    if (!evs.empty()) h0->evpool.push_back(evs.back());
    return st;
}

// S and N of several problems (one device, each handle on its own stream) with one
// persistent launch over a global tile queue, on hs[0]'s stream; synchronises that stream.
// The tile edge is the first handle's.
bem_status launch_assemble_batch(bem_ctx** hs, int nprob) {
    const int T = asm_tile_of(hs[0]);
    if (T == 15) return assemble_batch_tiles<15>(hs, nprob);
    if (T == 23) return assemble_batch_tiles<23>(hs, nprob);
    return assemble_batch_tiles<31>(hs, nprob);
}

// ---------------------------------------------------------------------------------------
// plane-wave right-hand sides
//   per segment e and direction d: beta = k h_e (d.t_e), base = exp(i k d.P0_e),
//   phi_0 = int_0^1 (1-s) e^{i beta s} ds = sum_n (i beta)^n / (n! (n+1)(n+2)),
//   phi_1 = int_0^1 s e^{i beta s} ds     = sum_n (i beta)^n / (n! (n+2))
//   f-part  -i k (d.nu_e) h_e base phi_a   (f_i = -<phi_i, du/dnu>)
//   h2-part h_e base phi_a                  ([h2]_i = <phi_i, u_inc>)
// ---------------------------------------------------------------------------------------
// e^{i x} in double-float: x = n pi/2 + r, |r| <= pi/4 (n pi/2 formed as a double-float
// product, good to about 1e-15 |x| for the phases met here), Taylor series of sin r and
// cos r to r^21 (truncation below 1e-19), then the quadrant.
__device__ __forceinline__ void dfl_sincos(dfl x, dfl& sn, dfl& cs) {
    const float nf = rintf(x.hi * 0.636619772367581f);
    const dfl r = dfl_sub(x, dfl_mul(dfl{nf, 0.f}, dfl_mk(c_pio2_df)));
    const dfl r2 = dfl_mul(r, r);
    dfl ps = dfl_mk(c_sin_df[SC_TERMS - 1]), pc = dfl_mk(c_cos_df[SC_TERMS - 1]);
#pragma unroll
    for (int j = SC_TERMS - 2; j >= 0; --j) {
        ps = dfl_fma(ps, r2, dfl_mk(c_sin_df[j]));
        pc = dfl_fma(pc, r2, dfl_mk(c_cos_df[j]));
    }
    const dfl s0 = dfl_mul(ps, r), c0 = pc;
    switch (((int)nf) & 3) {
        case 0: sn = s0; cs = c0; break;
        case 1: sn = c0; cs = dfl_neg(s0); break;
        case 2: sn = dfl_neg(s0); cs = dfl_neg(c0); break;
        default: sn = dfl_neg(c0); cs = s0; break;
    }
}

// Per segment e and direction d (all in double-float on the FP32 pipe):
//   beta = k h_e (d.t_e), base = h_e exp(i k d.P0_e),
//   phi_0 = int_0^1 (1-s) e^{i beta s} ds = sum_n (i beta)^n / (n! (n+1)(n+2)),
//   phi_1 = int_0^1 s e^{i beta s} ds     = sum_n (i beta)^n / (n! (n+2))
//   f-part  -i k (d.nu_e) base phi_a                (f_i = -<phi_i, du/dnu>)
//   h2-part base phi_a                              ([h2]_i = <phi_i, u_inc>)
__global__ void __launch_bounds__(256) k_rhs(const double* seg, int N, const double* angles, double k,
                                             cplx* f, cplx* hz, int64_t ld) {
    // a CTA writes 255 vertices from the 256 segments around them (one per thread)
    __shared__ float4 sf0[256], sf1[256], sh0[256], sh1[256];
    __shared__ float2 s_d[3];                 // d_x, d_y, k (double-float)
    const int i0 = blockIdx.x * 255, w = blockIdx.y;
    if (threadIdx.x == 0) {
        double dy_, dx_;
        sincos(angles[w], &dy_, &dx_);
        const dfl a = dfl_from(dx_), b = dfl_from(dy_), c = dfl_from(k);
        s_d[0] = make_float2(a.hi, a.lo); s_d[1] = make_float2(b.hi, b.lo); s_d[2] = make_float2(c.hi, c.lo);
    }
    __syncthreads();
    const dfl dxd = dfl_mk(s_d[0]), dyd = dfl_mk(s_d[1]), kd = dfl_mk(s_d[2]);
    {
        const int t = threadIdx.x;
        int e = i0 - 1 + t;                   // in [-1, N + 254]: wrapped by adding or subtracting N
        while (e < 0) e += N;
        while (e >= N) e -= N;
        const dfl x0 = dfl_from_bits(seg[e]), y0 = dfl_from_bits(seg[N + e]);
        const dfl tx = dfl_from_bits(seg[2 * N + e]), ty = dfl_from_bits(seg[3 * N + e]);
        const dfl he = dfl_from_bits(seg[4 * N + e]);
        const dfl beta = dfl_mul(dfl_mul(kd, he), dfl_fma(dxd, tx, dfl_mul(dyd, ty)));
        const dfl dn = dfl_sub(dfl_mul(dxd, ty), dfl_mul(dyd, tx));          // d . nu_e, nu = (ty, -tx)
        dfl sb, cb;
        dfl_sincos(dfl_mul(kd, dfl_fma(dxd, x0, dfl_mul(dyd, y0))), sb, cb);
        // series: c = (i beta)^n / n!
        cdfl c = {{1.f, 0.f}, {0.f, 0.f}}, p0 = cdfl_zero(), p1 = cdfl_zero();
        for (int n = 0; n < RCP_MAX - 2; ++n) {
            const dfl r1 = dfl_mk(c_rcp_df[n + 1]), r2 = dfl_mk(c_rcp_df[n + 2]);
            const dfl r12 = dfl_mul(r1, r2);
            p0 = cdfl_fma_real(r12, c, p0);
            p1 = cdfl_fma_real(r2, c, p1);
            // c <- c * i beta / (n+1)
            const dfl br = dfl_mul(beta, r1);
            const cdfl nc = {dfl_neg(dfl_mul(c.im, br)), dfl_mul(c.re, br)};
            c = nc;
            if (fabsf(c.re.hi) + fabsf(c.im.hi) < 1e-19f) break;
        }
        const cdfl base = {dfl_mul(cb, he), dfl_mul(sb, he)};
        auto cmul_df = [](const cdfl& a, const cdfl& b) -> cdfl {
            return {dfl_fma(a.re, b.re, dfl_neg(dfl_mul(a.im, b.im))), dfl_fma(a.re, b.im, dfl_mul(a.im, b.re))};
        };
        const cdfl b0 = cmul_df(base, p0), b1 = cmul_df(base, p1);
        // -i k dn * b = (k dn b.im, -k dn b.re)
        const dfl kdn = dfl_mul(kd, dn);
        sf0[t] = cdfl_pack({dfl_mul(kdn, b0.im), dfl_neg(dfl_mul(kdn, b0.re))});
        sf1[t] = cdfl_pack({dfl_mul(kdn, b1.im), dfl_neg(dfl_mul(kdn, b1.re))});
        sh0[t] = cdfl_pack(b0);
        sh1[t] = cdfl_pack(b1);
    }
    __syncthreads();
    const int i = i0 + threadIdx.x;
    if (threadIdx.x >= 255 || i >= N) return;
    const int t = threadIdx.x;
    // vertex i: segment i (local t+1) as node 0, segment i-1 (local t) as node 1
    if (f) f[(int64_t)i + (int64_t)w * ld] = cdfl_to(cdfl_add(cdfl_unpack(sf0[t + 1]), cdfl_unpack(sf1[t])));
    if (hz) hz[(int64_t)i + (int64_t)w * ld] = cdfl_to(cdfl_add(cdfl_unpack(sh0[t + 1]), cdfl_unpack(sh1[t])));
}

bem_status launch_rhs(bem_ctx* h, const double* angles, int64_t nrhs, cplx* f, cplx* hz, int64_t ld) {
    dim3 grid((unsigned)((h->N + 254) / 255), (unsigned)nrhs);
    BEM_TIMED(h, "k_rhs", (k_rhs<<<grid, 256, 0, h->stream>>>(h->seg, (int)h->N, angles, h->k, f, hz, ld)));
    BEM_LAUNCH(h, "k_rhs");
    return BEM_OK;
}

// ---------------------------------------------------------------------------------------
// line-source right-hand sides: u_inc(x) = g2(|x - r0|) = (i/4) H0^(1)(k |x - r0|), the field
// of a z-directed line source at r0 (the 2D source of the TE problem), with
//   d u_inc / d nu = -(i k / 4) H1^(1)(k rho) (x - r0).nu / rho,  rho = |x - r0|,
//   f_i = -<phi_i, d u_inc / d nu>,  [h2]_i = <phi_i, u_inc>,
// by 8-point Gauss-Legendre on each segment (the source lies off the curve, at a distance of
// many segment lengths, so the integrand is smooth there).  One thread per vertex i and
// source w: segment i carries lambda_0 = 1 - s, segment i - 1 carries lambda_1 = s.
// ---------------------------------------------------------------------------------------
#define PS_Q 8
__global__ void __launch_bounds__(256) k_rhs_point(const double* __restrict__ seg, int N,
                                                   const double* __restrict__ src, double k, cplx* f, cplx* hz,
                                                   int64_t ld) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (i >= N) return;
    const double sx = src[2 * w], sy = src[2 * w + 1];
    double fr = 0.0, fi = 0.0, hr = 0.0, hi = 0.0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int e = side == 0 ? i : (i == 0 ? N - 1 : i - 1);
        const double x0 = seg[e], y0 = seg[N + e], tx = seg[2 * N + e], ty = seg[3 * N + e], he = seg[4 * N + e];
        for (int j = 0; j < PS_Q; ++j) {
            const double s = c_glx[gl_off(PS_Q) + j];
            const double lam = side == 0 ? 1.0 - s : s;
            const double wl = c_glw[gl_off(PS_Q) + j] * lam * he;
            const double dx = x0 + s * he * tx - sx, dy = y0 + s * he * ty - sy;
            const double rho = sqrt(dx * dx + dy * dy);
            const Bessel01 b = bessel01<true>(k * rho);
            // u = (i/4)(J0 + i Y0) ;  du/dnu = -(i k/4)(J1 + i Y1) (d.nu)/rho = (k/4)(Y1 - i J1) (d.nu)/rho
            const double dn = (dx * ty - dy * tx) / rho;
            hr += wl * (-0.25 * b.Y0);
            hi += wl * (0.25 * b.J0);
            fr -= wl * (0.25 * k * b.Y1 * dn);
            fi -= wl * (-0.25 * k * b.J1 * dn);
        }
    }
    if (f) f[(int64_t)i + (int64_t)w * ld] = cmk(fr, fi);
    if (hz) hz[(int64_t)i + (int64_t)w * ld] = cmk(hr, hi);
}

bem_status launch_rhs_point(bem_ctx* h, const double* src, int64_t nsrc, cplx* f, cplx* hz, int64_t ld) {
    dim3 grid((unsigned)((h->N + 255) / 256), (unsigned)nsrc);
    BEM_TIMED(h, "k_rhs_point", (k_rhs_point<<<grid, 256, 0, h->stream>>>(h->seg, (int)h->N, src, h->k, f, hz, ld)));
    BEM_LAUNCH(h, "k_rhs_point");
    return BEM_OK;
}

// =======================================================================================
// Shape gradient (vector-Jacobian products of the assembly, the right-hand sides and the
// Gram matrix with respect to the vertex coordinates).  For complex weights Omega (N x N,
// passed transposed: OmT[j + i N] = Omega_ij) the pair kernel accumulates
//     grad += d/d verts  Re sum_ij (Omega^S_ij S_ij + Omega^W_ij N_ij),
// differentiating each segment pair's integrals: separated pairs by differentiating the
// Gauss rule (dg/dr = -(i/4) k H1(k r), the node positions and the chord lengths), self
// pairs through the closed form in h, adjacent pairs through the Duffy nodes (the closed
// rho integrals are functions of |R(w)|^2).  FP64.  Each unordered pair {e, f} is visited
// once; the two orderings share the integrals (I^{fe}_{ba} = I^{ef}_{ab}).
// =======================================================================================
struct VjpParams {
    int N;
    double k;
    const double* seg;
    const double* btab;
    SeriesCoef sc;
    const cplx* OmS;     // transposed: OmS[j + i N] = Omega^S_ij
    const cplx* OmW;
    double* grad;        // 2N: (x_i, y_i)
};

__device__ __forceinline__ cplx om_at(const cplx* OmT, int N, int i, int j) { return OmT[(int64_t)j + (int64_t)i * N]; }

// the four pair weights w_ab (a: node on e, b: node on f), both orderings folded in
__device__ __forceinline__ void pair_weights(const cplx* OmT, int N, int e, int f, bool self, cplx w[4]) {
    const int ie[2] = {e, (e + 1) % N}, jf[2] = {f, (f + 1) % N};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            cplx v = om_at(OmT, N, ie[a], jf[b]);
            if (!self) v = cadd(v, om_at(OmT, N, jf[b], ie[a]));
            w[a * 2 + b] = v;
        }
}

__device__ __forceinline__ double re_mul(cplx a, cplx b) { return a.x * b.x - a.y * b.y; }   // Re(a b)

// self pair: I_ab(h) closed form and dI_ab/dh
__device__ void pair_self_dh(double h, const SeriesCoef& sc, cplx I[4], cplx dI[4]) {
    const double lnh = log(h);
    cplx i11 = cmk(0, 0), i01 = cmk(0, 0), d11 = cmk(0, 0), d01 = cmk(0, 0);
    double h2m = h * h;                 // h^{2m+2}
    for (int m = 0; m < sc.nm; ++m) {
        const double p = 2.0 * m;
        const double T11 = (2.0 / 3.0) / (p + 1) - 1.0 / (p + 2) + (1.0 / 3.0) / (p + 4);
        const double L11 = -(2.0 / 3.0) / ((p + 1) * (p + 1)) + 1.0 / ((p + 2) * (p + 2)) -
                           (1.0 / 3.0) / ((p + 4) * (p + 4));
        const double T01 = (1.0 / 3.0) / (p + 1) - (1.0 / 3.0) / (p + 4);
        const double L01 = -(1.0 / 3.0) / ((p + 1) * (p + 1)) + (1.0 / 3.0) / ((p + 4) * (p + 4));
        const cplx A = sc.A[m];
        const double B = sc.B[m];
        const cplx f11 = cmk(A.x * T11 + B * (lnh * T11 + L11), A.y * T11);
        const cplx f01 = cmk(A.x * T01 + B * (lnh * T01 + L01), A.y * T01);
        i11 = cadd(i11, cscale(f11, h2m));
        i01 = cadd(i01, cscale(f01, h2m));
        // d/dh [h^{2m+2} f(ln h)] = h^{2m+1} [(2m+2) f + B T]
        const double h2m1 = h2m / h;
        d11 = cadd(d11, cscale(cmk((p + 2.0) * f11.x + B * T11, (p + 2.0) * f11.y), h2m1));
        d01 = cadd(d01, cscale(cmk((p + 2.0) * f01.x + B * T01, (p + 2.0) * f01.y), h2m1));
        h2m *= h * h;
    }
    I[0] = i11; I[3] = i11; I[1] = i01; I[2] = i01;
    dI[0] = d11; dI[3] = d11; dI[1] = d01; dI[2] = d01;
}

// G_j(R2) of the adjacent-pair rho integrals and dG_j/dR2 (the series of adjacent_node)
__device__ void adj_G(double R2, const SeriesCoef& sc, cplx G[3], cplx dG[3]) {
    const double lnR = 0.5 * log(R2);
    for (int j = 0; j < 3; ++j) { G[j] = cmk(0, 0); dG[j] = cmk(0, 0); }
    double R2m = 1.0;
    for (int m = 0; m < sc.nm; ++m) {
        for (int j = 0; j < 3; ++j) {
            const double a = 2.0 + j + 2.0 * m;
            const cplx term = cmk((sc.A[m].x + sc.B[m] * lnR) / a - sc.B[m] / (a * a), sc.A[m].y / a);
            G[j] = cadd(G[j], cscale(term, R2m));
            // d/dR2 [R2^m term(lnR)] = m R2^{m-1} term + R2^m B/(2 a R2)
            const double dr = (m > 0 ? m * R2m / R2 : 0.0);
            dG[j] = cadd(dG[j], cmk(dr * term.x + R2m * sc.B[m] / (2.0 * a * R2), dr * term.y));
        }
        R2m *= R2;
    }
}

__global__ void __launch_bounds__(256) k_assemble_vjp(VjpParams p) {
    const int N = p.N;
    const int e = blockIdx.y;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d > N / 2) return;
    if ((N % 2) == 0 && d == N / 2 && e >= N / 2) return;    // each unordered pair once
    const int f = (e + d) % N;
    const SegV se = load_seg(p.seg, N, e), sf = load_seg(p.seg, N, f);
    cplx wS[4], wW[4];
    pair_weights(p.OmS, N, e, f, d == 0, wS);
    pair_weights(p.OmW, N, e, f, d == 0, wW);
    const double k2 = p.k * p.k;
    const double sg[2] = {-1.0, 1.0};
    cplx wM = cmk(0, 0);                        // sum_ab wW_ab sigma_a sigma_b (Maue's M0 term)
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) wM = cadd(wM, cscale(wW[a * 2 + b], sg[a] * sg[b]));
    double g[8] = {0, 0, 0, 0, 0, 0, 0, 0};     // d/d (x_e, y_e, x_e+1, y_e+1, x_f, y_f, x_f+1, y_f+1)
    if (d == 0) {
        // self pair: a function of h_e only
        cplx I[4], dI[4];
        const double h = se.h;
        pair_self_dh(h, p.sc, I, dI);
        const cplx sI = cadd(cadd(I[0], I[1]), cadd(I[2], I[3]));
        const cplx sdI = cadd(cadd(dI[0], dI[1]), cadd(dI[2], dI[3]));
        double rho = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const int ab = a * 2 + b;
                // N_ab = sigma_a sigma_b sum I / h^2 - k^2 I_ab
                const cplx dW = csub(cscale(csub(cscale(sdI, 1.0 / (h * h)), cscale(sI, 2.0 / (h * h * h))), sg[a] * sg[b]),
                                     cscale(dI[ab], k2));
                rho += re_mul(wS[ab], dI[ab]) + re_mul(wW[ab], dW);
            }
        g[0] -= rho * se.tx; g[1] -= rho * se.ty;
        g[2] += rho * se.tx; g[3] += rho * se.ty;
    } else {
        const double hh = se.h * sf.h;
        const double c = se.tx * sf.tx + se.ty * sf.ty;              // nu_e . nu_f = t_e . t_f
        cplx kap[4];
        for (int ab = 0; ab < 4; ++ab)
            kap[ab] = cadd(cscale(csub(wS[ab], cscale(wW[ab], k2 * c)), hh), wM);
        cplx A[4] = {cmk(0, 0), cmk(0, 0), cmk(0, 0), cmk(0, 0)};  // I_ab / (h_e h_f)
        if (d == 1) {
            // adjacent pair (f = e + 1): vertices P_A = x_e, P_B = x_e+1, P_C = x_e+2;
            // R = dE + w dF (tri 0) or w dE + dF (tri 1), dE = P_B - P_A, dF = P_C - P_B
            const int qw = 16;
            const double dEx = se.h * se.tx, dEy = se.h * se.ty, dFx = sf.h * sf.tx, dFy = sf.h * sf.ty;
            double gA[2] = {0, 0}, gB[2] = {0, 0}, gC[2] = {0, 0};
            for (int tri = 0; tri < 2; ++tri) {
                for (int iw = 0; iw < qw; ++iw) {
                    const double w = c_glx[gl_off(qw) + iw], ww = c_glw[gl_off(qw) + iw];
                    double cc[4][3];
                    double Rx, Ry, dA, dB, dC;       // dR/dP_A, dR/dP_B, dR/dP_C (scalar multiples of I)
                    if (tri == 0) {
                        Rx = dEx + w * dFx; Ry = dEy + w * dFy;
                        dA = -1.0; dB = 1.0 - w; dC = w;
                        cc[0][0] = 0; cc[0][1] = 1; cc[0][2] = -w;
                        cc[1][0] = 0; cc[1][1] = 0; cc[1][2] = w;
                        cc[2][0] = 1; cc[2][1] = -(1 + w); cc[2][2] = w;
                        cc[3][0] = 0; cc[3][1] = w; cc[3][2] = -w;
                    } else {
                        Rx = w * dEx + dFx; Ry = w * dEy + dFy;
                        dA = -w; dB = w - 1.0; dC = 1.0;
                        cc[0][0] = 0; cc[0][1] = w; cc[0][2] = -w;
                        cc[1][0] = 0; cc[1][1] = 0; cc[1][2] = w;
                        cc[2][0] = 1; cc[2][1] = -(1 + w); cc[2][2] = w;
                        cc[3][0] = 0; cc[3][1] = 1; cc[3][2] = -w;
                    }
                    cplx G[3], dG[3];
                    adj_G(Rx * Rx + Ry * Ry, p.sc, G, dG);
                    cplx xi = cmk(0, 0);
                    for (int ab = 0; ab < 4; ++ab) {
                        cplx sG = cmk(0, 0), sdG = cmk(0, 0);
                        for (int j = 0; j < 3; ++j) {
                            sG = cadd(sG, cscale(G[j], cc[ab][j]));
                            sdG = cadd(sdG, cscale(dG[j], cc[ab][j]));
                        }
                        A[ab] = cadd(A[ab], cscale(sG, ww));
                        xi = cadd(xi, cmul(kap[ab], cscale(sdG, ww)));
                    }
                    // d|R|^2 = 2 R . dR
                    const double r2c = 2.0 * xi.x;
                    gA[0] += r2c * dA * Rx; gA[1] += r2c * dA * Ry;
                    gB[0] += r2c * dB * Rx; gB[1] += r2c * dB * Ry;
                    gC[0] += r2c * dC * Rx; gC[1] += r2c * dC * Ry;
                }
            }
            // chord lengths and the tangent product
            double hpart = 0.0, cpart = 0.0;
            for (int ab = 0; ab < 4; ++ab) {
                hpart += re_mul(csub(wS[ab], cscale(wW[ab], k2 * c)), A[ab]);
                cpart += -k2 * hh * re_mul(wW[ab], A[ab]);
            }
            const double ce[2] = {(sf.tx - c * se.tx) / se.h, (sf.ty - c * se.ty) / se.h};   // dc/dP_B via t_e
            const double cf[2] = {(se.tx - c * sf.tx) / sf.h, (se.ty - c * sf.ty) / sf.h};   // dc/dP_C via t_f
            const double te[2] = {se.tx, se.ty}, tf[2] = {sf.tx, sf.ty};
            for (int q = 0; q < 2; ++q) {
                gA[q] += hpart * (-sf.h * te[q]) + cpart * (-ce[q]);
                gB[q] += hpart * (sf.h * te[q] - se.h * tf[q]) + cpart * (ce[q] - cf[q]);
                gC[q] += hpart * (se.h * tf[q]) + cpart * cf[q];
            }
            g[0] = gA[0]; g[1] = gA[1]; g[2] = gB[0]; g[3] = gB[1]; g[6] = gC[0]; g[7] = gC[1];
        } else {
            // separated pair: q x q Gauss, as in the assembly
            const float mx = (float)(se.x0 - sf.x0) + 0.5f * (float)(se.h * se.tx - sf.h * sf.tx);
            const float my = (float)(se.y0 - sf.y0) + 0.5f * (float)(se.h * se.ty - sf.h * sf.ty);
            const float hmax = (float)fmax(se.h, sf.h);
            const float gap = fmaxf(sqrtf(mx * mx + my * my) - 0.5f * (float)(se.h + sf.h), 0.0f);
            const int q = q_for_gap(gap / hmax, (float)p.k * (gap + hmax));
            const double* xs = c_glx + gl_off(q);
            const double* ws = c_glw + gl_off(q);
            const double ux = se.h * se.tx, uy = se.h * se.ty, vx = sf.h * sf.tx, vy = sf.h * sf.ty;
            for (int i = 0; i < q; ++i) {
                const double s = xs[i];
                const double px = se.x0 + s * ux, py = se.y0 + s * uy;
                for (int j = 0; j < q; ++j) {
                    const double t = xs[j], wgt = ws[i] * ws[j];
                    const double Dx = sf.x0 + t * vx - px, Dy = sf.y0 + t * vy - py;
                    const BesselU bu = bessel_u<true>(p.btab, k2 * (Dx * Dx + Dy * Dy));
                    const cplx gv = cmk(-0.25 * bu.Y0, 0.25 * bu.J0);                  // (i/4) H0
                    const cplx gq = cmk(0.25 * k2 * bu.Y1z, -0.25 * k2 * bu.J1z);      // g'(r)/r
                    const double la[2] = {1.0 - s, s}, lb[2] = {1.0 - t, t};
                    cplx kp = cmk(0, 0);
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            const double l = la[a] * lb[b];
                            A[a * 2 + b] = cadd(A[a * 2 + b], cscale(gv, wgt * l));
                            kp = cadd(kp, cscale(kap[a * 2 + b], l));
                        }
                    const double co = wgt * re_mul(kp, gq);
                    // r dr/dx_e = -(1-s) D, r dr/dx_e+1 = -s D, r dr/dx_f = (1-t) D, r dr/dx_f+1 = t D
                    g[0] -= co * (1.0 - s) * Dx; g[1] -= co * (1.0 - s) * Dy;
                    g[2] -= co * s * Dx;         g[3] -= co * s * Dy;
                    g[4] += co * (1.0 - t) * Dx; g[5] += co * (1.0 - t) * Dy;
                    g[6] += co * t * Dx;         g[7] += co * t * Dy;
                }
            }
            double hpart = 0.0, cpart = 0.0;
            for (int ab = 0; ab < 4; ++ab) {
                hpart += re_mul(csub(wS[ab], cscale(wW[ab], k2 * c)), A[ab]);
                cpart += -k2 * hh * re_mul(wW[ab], A[ab]);
            }
            const double te[2] = {se.tx, se.ty}, tf[2] = {sf.tx, sf.ty};
            for (int q2 = 0; q2 < 2; ++q2) {
                const double ce = (tf[q2] - c * te[q2]) / se.h, cf = (te[q2] - c * tf[q2]) / sf.h;
                g[0 + q2] += hpart * (-sf.h * te[q2]) - cpart * ce;
                g[2 + q2] += hpart * (sf.h * te[q2]) + cpart * ce;
                g[4 + q2] += hpart * (-se.h * tf[q2]) - cpart * cf;
                g[6 + q2] += hpart * (se.h * tf[q2]) + cpart * cf;
            }
        }
    }
    const int v[4] = {e, (e + 1) % N, f, (f + 1) % N};
    for (int q = 0; q < 4; ++q) {
        if (g[2 * q] != 0.0) atomicAdd(p.grad + 2 * v[q], g[2 * q]);
        if (g[2 * q + 1] != 0.0) atomicAdd(p.grad + 2 * v[q] + 1, g[2 * q + 1]);
    }
}

// Right-hand-side vector-Jacobian product: f_i(d) = sum over the two segments at vertex i
// of T_a = -i k (d x Delta) e^{i k d.x_e} phi_a(beta), beta = k d.Delta, Delta = x_e+1 - x_e
// (d x Delta = d_x Delta_y - d_y Delta_x = h_e (d . nu_e)), phi_0 = int (1-s) e^{i beta s},
// phi_1 = int s e^{i beta s}; grad += d/dverts Re sum_{i,w} om[i + w ld] f_i(d_w).
// One thread per (segment, direction).
__global__ void __launch_bounds__(256) k_rhs_vjp(const double* seg, int N, const double* angles, int nang, double k,
                                                  const cplx* om, int64_t ld, double* grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (e >= N || w >= nang) return;
    double dy_, dx_;
    sincos(angles[w], &dy_, &dx_);
    const SegV s = load_seg(seg, N, e);
    const double Dx = s.h * s.tx, Dy = s.h * s.ty;
    const double beta = k * (dx_ * Dx + dy_ * Dy);
    const double cr = dx_ * Dy - dy_ * Dx;
    // phi_a(beta) and phi_a'(beta): sums of (i beta)^n / n! times 1/((n+1)(n+2)), 1/(n+2);
    // derivatives i sum (i beta)^n/n! times 1/((n+2)(n+3)), 1/(n+3)
    cplx c = cmk(1, 0), p0 = cmk(0, 0), p1 = cmk(0, 0), q0 = cmk(0, 0), q1 = cmk(0, 0);
    for (int n = 0; n < 60; ++n) {
        const double a = n + 1.0, b = n + 2.0, cc = n + 3.0;
        p0 = cadd(p0, cscale(c, 1.0 / (a * b)));
        p1 = cadd(p1, cscale(c, 1.0 / b));
        q0 = cadd(q0, cscale(c, 1.0 / (b * cc)));
        q1 = cadd(q1, cscale(c, 1.0 / cc));
        c = cmul(c, cmk(0.0, beta / a));           // (i beta)^{n+1}/(n+1)!
        if (fabs(c.x) + fabs(c.y) < 1e-20) break;
    }
    q0 = cmul(cmk(0, 1), q0);
    q1 = cmul(cmk(0, 1), q1);
    double sp, cp;
    sincos(k * (dx_ * s.x0 + dy_ * s.y0), &sp, &cp);
    const cplx E = cmk(cp, sp);
    const cplx mik = cmk(0, -k);                 // -i k
    const cplx o0 = om[(int64_t)e + (int64_t)w * ld], o1 = om[(int64_t)((e + 1) % N) + (int64_t)w * ld];
    double gE[2] = {0, 0}, gE1[2] = {0, 0};
    const cplx phi[2] = {p0, p1}, dphi[2] = {q0, q1}, oo[2] = {o0, o1};
    for (int a = 0; a < 2; ++a) {
        const cplx pre = cmul(oo[a], cmul(mik, E));          // om * (-i k) e^{i k d.x_e}
        const cplx T = cmul(pre, cscale(phi[a], cr));         // om T_a
        // d/dDelta: (-d_y, d_x) phi + cr phi' k d ; d/dx_e (phase): i k d T
        const double gDx = re_mul(pre, cadd(cscale(phi[a], -dy_), cscale(dphi[a], cr * k * dx_)));
        const double gDy = re_mul(pre, cadd(cscale(phi[a], dx_), cscale(dphi[a], cr * k * dy_)));
        const cplx ikT = cmul(cmk(0, k), T);
        gE[0] += ikT.x * dx_ - gDx; gE[1] += ikT.x * dy_ - gDy;
        gE1[0] += gDx; gE1[1] += gDy;
    }
    atomicAdd(grad + 2 * e, gE[0]);
    atomicAdd(grad + 2 * e + 1, gE[1]);
    atomicAdd(grad + 2 * ((e + 1) % N), gE1[0]);
    atomicAdd(grad + 2 * ((e + 1) % N) + 1, gE1[1]);
}

// Gram-matrix term: G_ii = (h_i-1 + h_i)/3, G_i,i+1 = h_i/6, so for a pair (p, q) of
// N x nrhs blocks d/dh_e Re sum_r p_r^H G q_r = Re sum_r [(conj p_e q_e + conj p_e+1 q_e+1)/3
// + (conj p_e q_e+1 + conj p_e+1 q_e)/6]; with h_e = |x_e+1 - x_e| this moves grad by
// +-coef t_e.  Four signed pairs per call (sign[k] = 0 skips).
__global__ void k_gram_vjp(const double* seg, int N, int nrhs, const cplx* const* P, const cplx* const* Q,
                           const double* sign, double* grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int e1 = (e + 1) % N;
    double coef = 0.0;
    for (int t = 0; t < 4; ++t) {
        if (sign[t] == 0.0) continue;
        double acc = 0.0;
        for (int r = 0; r < nrhs; ++r) {
            const cplx pe = P[t][e + (int64_t)r * N], pe1 = P[t][e1 + (int64_t)r * N];
            const cplx qe = Q[t][e + (int64_t)r * N], qe1 = Q[t][e1 + (int64_t)r * N];
            const cplx d = cadd(cscale(cadd(cmul(cconj(pe), qe), cmul(cconj(pe1), qe1)), 1.0 / 3.0),
                                cscale(cadd(cmul(cconj(pe), qe1), cmul(cconj(pe1), qe)), 1.0 / 6.0));
            acc += d.x;
        }
        coef += sign[t] * acc;
    }
    const double tx = seg[2 * N + e], ty = seg[3 * N + e];
    atomicAdd(grad + 2 * e1, coef * tx);
    atomicAdd(grad + 2 * e1 + 1, coef * ty);
    atomicAdd(grad + 2 * e, -coef * tx);
    atomicAdd(grad + 2 * e + 1, -coef * ty);
}

bem_status launch_assemble_vjp(bem_ctx* h, const cplx* OmS, const cplx* OmW, double* grad) {
    if (h->N < 5) return bem_fail(h, BEM_E_UNSUPPORTED, "shape gradient: N >= 5 required");
    VjpParams p;
    p.N = (int)h->N;
    p.k = h->k;
    p.seg = h->seg;
    const float4* tabf = nullptr;
    bem_status st = bessel_table(h, &p.btab, &tabf);
    if (st != BEM_OK) return st;
    series_coefficients(h->k, 2.0 * (h->general ? h->hmax : h->hbar), &p.sc);
    p.OmS = OmS;
    p.OmW = OmW;
    p.grad = grad;
    dim3 grid((unsigned)((h->N / 2 + 1 + 255) / 256), (unsigned)h->N);
    BEM_TIMED(h, "k_assemble_vjp", (k_assemble_vjp<<<grid, 256, 0, h->stream>>>(p)));
    BEM_LAUNCH(h, "k_assemble_vjp");
    return BEM_OK;
}

bem_status launch_rhs_vjp(bem_ctx* h, const double* angles, int64_t nang, const cplx* om, int64_t ld, double* grad) {
    dim3 grid((unsigned)((h->N + 255) / 256), (unsigned)nang);
    BEM_TIMED(h, "k_rhs_vjp", (k_rhs_vjp<<<grid, 256, 0, h->stream>>>(h->seg, (int)h->N, angles, (int)nang, h->k, om, ld, grad)));
    BEM_LAUNCH(h, "k_rhs_vjp");
    return BEM_OK;
}

bem_status launch_gram_vjp(bem_ctx* h, int nrhs, const cplx* const* P_dev, const cplx* const* Q_dev,
                           const double* sign_dev, double* grad) {
    BEM_TIMED(h, "k_gram_vjp", (k_gram_vjp<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(
                                    h->seg, (int)h->N, nrhs, P_dev, Q_dev, sign_dev, grad)));
    BEM_LAUNCH(h, "k_gram_vjp");
    return BEM_OK;
}
