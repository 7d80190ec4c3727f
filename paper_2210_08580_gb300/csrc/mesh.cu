// Non-equal-chord meshes.  Sec. III-A builds the filter of a non-homogeneous discretisation
// from the orthonormalised Laplacian L~ = G^-1/2 L G^-1/2 instead of L.  On such a polygon the
// P1 Gram matrix G and Laplacian L are general cyclic tridiagonal matrices,
//     G_ii = (h_{i-1} + h_i)/3,  G_{i,i+1} = h_i/6;   L_ii = 1/h_{i-1} + 1/h_i,  L_{i,i+1} = -1/h_i
// (segment i runs from vertex i to i+1), so neither is diagonalised by Fourier modes.  This
// file supplies what the equal-chord path gets from circulant algebra:
//
//  * exact solves with G (and with L + sigma G) through a bordered LDL^T factorisation:
//    the first N-1 unknowns form a tridiagonal block factored without fill, the last
//    unknown is the border; T = L D L^T with L unit lower bidiagonal plus a dense last row.
//    With F = D^1/2 L^T, F^T F = G, the factor the compression needs (B^ = B F^-1 has the
//    singular values and left singular vectors of B G^-1/2).
//  * the filter basis Phi (N x n, G-orthonormal): the eigenvectors of the n lowest
//    eigenvalues of the pencil L phi = lambda G phi.  In the x-coordinates j2 = G^1/2 x the
//    filter P^L_n = V_n V_n^T (V_n the lowest eigenvectors of L~) reads P_x = Phi Phi^T G
//    with Phi = G^-1/2 V_n, so the filtered compact part is P_x C_x = Phi B with
//        B = Phi^T G C_x = (Phi^T S) G^-1 N - (G Phi)^T / 4 - alpha Phi^T D.
//    Only span(Phi) matters (any orthogonal mixing of its columns cancels in Phi B and in the
//    compression), so Phi is found by Chebyshev-accelerated shift-and-invert subspace
//    iteration on sigma (L + sigma G)^-1 G from the arclength Fourier modes, G-orthonormalised
//    every second step by a Cholesky QR, and one Rayleigh-Ritz step at the end whose small
//    eigenproblem runs through the library's one-sided Jacobi SVD.  Its dense products and
//    the small Cholesky run in double-float on the FP32 pipe.
#include <math.h>

#include <algorithm>
#include <vector>

#include "dfloat.cuh"
#include "kernels.h"

// Chunks of the chunked solves: forward chunk c covers i in [1 + c CL, 1 + (c+1) CL) within
// [1, N-1); backward chunk c covers i from N-3 - c CL down to N-2 - (c+1) CL within [0, N-2).
#define CYC_CL 64
#define CYC_FAC 7
#define CYC_PF 16                     // elements (chunks) a solve pass loads before computing
__host__ __device__ __forceinline__ int64_t cyc_nch(int64_t N) { return (N - 2 + CYC_CL - 1) / CYC_CL; }

// -----------------------------------------------------------------------------------------
// Bordered LDL^T of a cyclic symmetric tridiagonal matrix T with
//     T_ii = cL (1/h_{i-1} + 1/h_i) + cG (h_{i-1} + h_i)/3,
//     T_{i,i+1} = T_{i+1,i} = -cL / h_i + cG h_i / 6       (indices mod N)
// Factor layout (CYC_FAC N doubles): l[i] (i = 1..N-2, subdiagonal of L), dinv[i] = 1/d_i,
// m[i] (i = 0..N-2, L's last row), sdinv[i] = d_i^-1/2, then the chunk propagators of the
// chunked solves: psiF[i] = prod (-l_k) over k from i's forward chunk start to i,
// psiB[i] = prod (-l_{k+1}) over k from i's backward chunk top down to i, and per forward
// chunk c msum[c] = sum m_i psiF[i].
// -----------------------------------------------------------------------------------------
__device__ __forceinline__ double tri_diag(const double* h, int N, int i, double cL, double cG) {
    const double hp = h[i == 0 ? N - 1 : i - 1], hi = h[i];
    return cL * (1.0 / hp + 1.0 / hi) + cG * (hp + hi) * (1.0 / 3.0);
}
__device__ __forceinline__ double tri_off(const double* h, int i, double cL, double cG) {
    return -cL / h[i] + cG * h[i] * (1.0 / 6.0);
}

// coefficients for the factorisation: a (diagonal) in the sd slot, b (T_{i,i+1}) in the m slot
__global__ void k_tri_coef(const double* __restrict__ h, int N, double cL, double cG, double* fac) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    fac[3 * N + i] = tri_diag(h, N, i, cL, cG);
    fac[2 * N + i] = tri_off(h, i, cL, cG);
}

// -----------------------------------------------------------------------------------------
// The factorisation in parallel over chunks of CYC_CL pivots.  The pivots are ratios of
// leading minors, P_i = a_i P_{i-1} - b_{i-1}^2 P_{i-2}, d_i = P_i / P_{i-1}: each chunk's
// product of the 2 x 2 transfer matrices (rescaled by powers of two) is formed in parallel,
// one thread carries the minors' vector over the chunks, and each chunk then runs the pivot
// recursion from its carried start (a start off by rounding is pulled back by the recursion,
// whose derivative b^2/d^2 = l^2 is below one).  The border column z_i = c_0 prod (-l_k) is a
// prefix product, carried the same way, and the Schur complement is summed per chunk in a
// fixed order.  Scratch: 9 nch + 3 doubles in the msum slot (k_cyc_prop fills it afterwards).
// -----------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t fac_nch(int64_t N) { return (N - 1 + CYC_CL - 1) / CYC_CL; }

__device__ __forceinline__ double pow2_scale_of(double m) {      // 2^-e with m = f 2^e, f in [0.5, 1)
    int e;
    frexp(m, &e);
    return ldexp(1.0, -e);
}

__global__ void k_fac_transfer(int64_t N, double* fac) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nch = fac_nch(N);
    if (c >= nch) return;
    const double* b = fac + 2 * N;            // T_{i,i+1} (m slot, on entry)
    const double* a = fac + 3 * N;            // diagonal (sd slot, on entry)
    double* T = fac + 6 * N + 4 * c;
    double t00 = 1.0, t01 = 0.0, t10 = 0.0, t11 = 1.0;
    const int64_t s = c * CYC_CL, e = min(N - 1, s + CYC_CL);
    for (int64_t i = s; i < e; ++i) {
        const double bb = (i >= 1) ? b[i - 1] * b[i - 1] : 0.0;
        // [[a_i, -bb], [1, 0]] times T
        const double n00 = a[i] * t00 - bb * t10, n01 = a[i] * t01 - bb * t11;
        t10 = t00; t11 = t01; t00 = n00; t01 = n01;
        const double sc = pow2_scale_of(fmax(fmax(fabs(t00), fabs(t01)), fmax(fabs(t10), fabs(t11))));
        t00 *= sc; t01 *= sc; t10 *= sc; t11 *= sc;
    }
    T[0] = t00; T[1] = t01; T[2] = t10; T[3] = t11;
}

__global__ void k_fac_carry(int64_t N, double* fac) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t nch = fac_nch(N);
    const double* T = fac + 6 * N;
    double* v = fac + 6 * N + 4 * nch;
    double v0 = 1.0, v1 = 0.0;                // (P_{-1}, P_{-2})
    for (int64_t c = 0; c < nch; ++c) {
        v[2 * c] = v0; v[2 * c + 1] = v1;
        const double w0 = T[4 * c] * v0 + T[4 * c + 1] * v1, w1 = T[4 * c + 2] * v0 + T[4 * c + 3] * v1;
        const double sc = pow2_scale_of(fmax(fabs(w0), fabs(w1)));
        v0 = w0 * sc; v1 = w1 * sc;
    }
}

// pivots of chunk c from its carried minors, and the chunk's prefix products of (-l) (into the
// psiF slot) with their total
__global__ void k_fac_pivots(int64_t N, double* fac, int* err) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nch = fac_nch(N);
    if (c >= nch) return;
    double* l = fac;
    double* dinv = fac + N;
    const double* b = fac + 2 * N;
    double* a_sd = fac + 3 * N;
    double* loc = fac + 4 * N;
    const double* v = fac + 6 * N + 4 * nch;
    double* tot = fac + 6 * N + 6 * nch;
    const int64_t s = c * CYC_CL, e = min(N - 1, s + CYC_CL);
    double d = (c == 0) ? 0.0 : v[2 * c] / v[2 * c + 1];      // d_{s-1}
    double p = 1.0;
    bool bad = false;
    for (int64_t i = s; i < e; ++i) {
        double dn;
        if (i == 0) {
            dn = a_sd[0];
        } else {
            const double li = b[i - 1] / d;
            l[i] = li;
            dn = fma(-li, b[i - 1], a_sd[i]);
            p *= -li;
        }
        bad |= !(dn > 0.0);
        d = dn;
        const double di = 1.0 / dn;
        dinv[i] = di;
        a_sd[i] = sqrt(di);
        if (i <= N - 3) loc[i] = p;
    }
    tot[c] = p;
    if (bad) atomicOr(err, DEVERR_SINGULAR);
}

// z_in per chunk (one thread), then z, m and the Schur partials per chunk
__global__ void k_fac_border_carry(int64_t N, double* fac) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t nch = fac_nch(N);
    const double* b = fac + 2 * N;
    const double* tot = fac + 6 * N + 6 * nch;
    double* zin = fac + 6 * N + 7 * nch;
    double* ends = fac + 6 * N + 9 * nch;     // c_0, c_{N-2}, z_{N-3}
    ends[0] = b[N - 1];
    ends[1] = b[N - 2];
    double z = b[N - 1];
    for (int64_t c = 0; c < nch; ++c) {
        zin[c] = z;
        z *= tot[c];
    }
}

__global__ void k_fac_border(int64_t N, double* fac) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nch = fac_nch(N);
    if (c >= nch) return;
    const double* dinv = fac + N;
    double* m = fac + 2 * N;
    const double* loc = fac + 4 * N;
    const double* zin = fac + 6 * N + 7 * nch;
    double* part = fac + 6 * N + 8 * nch;
    double* ends = fac + 6 * N + 9 * nch;
    const int64_t s = c * CYC_CL, e = min(N - 2, s + CYC_CL);
    double sp = 0.0;
    for (int64_t i = s; i < e; ++i) {
        const double z = zin[c] * loc[i];
        m[i] = z * dinv[i];
        sp = fma(z * z, dinv[i], sp);
        if (i == N - 3) ends[2] = z;
    }
    part[c] = sp;
}

__global__ void k_fac_final(int64_t N, double* fac, int* err) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t nch = fac_nch(N);
    double* l = fac;
    double* dinv = fac + N;
    double* m = fac + 2 * N;
    double* a_sd = fac + 3 * N;
    const double* part = fac + 6 * N + 8 * nch;
    const double* ends = fac + 6 * N + 9 * nch;
    const double zl = ends[1] - l[N - 2] * ends[2];        // z_{N-2} = c_{N-2} - l_{N-2} z_{N-3}
    m[N - 2] = zl * dinv[N - 2];
    double schur = 0.0;
    for (int64_t c = 0; c < nch; ++c) schur += part[c];
    schur = fma(zl * zl, dinv[N - 2], schur);
    const double dl = a_sd[N - 1] - schur;
    if (!(dl > 0.0)) atomicOr(err, DEVERR_SINGULAR);
    l[0] = 0.0;
    l[N - 1] = 0.0;
    m[N - 1] = 0.0;
    dinv[N - 1] = 1.0 / dl;
    a_sd[N - 1] = sqrt(1.0 / dl);
}



__global__ void k_cyc_prop(int64_t N, double* fac) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cyc_nch(N)) return;
    const double* l = fac;
    const double* m = fac + 2 * N;
    double* psiF = fac + 4 * N;
    double* psiB = fac + 5 * N;
    double* msum = fac + 6 * N;
    double psi = 1.0, ms = 0.0;
    const int64_t s = 1 + c * CYC_CL, e = min(N - 1, s + CYC_CL);
    for (int64_t i = s; i < e; ++i) {
        psi *= -l[i];
        psiF[i] = psi;
        ms = fma(m[i], psi, ms);
    }
    msum[c] = ms;
    const int64_t t = N - 3 - c * CYC_CL, b = max((int64_t)0, t - CYC_CL + 1);
    double phi = 1.0;
    for (int64_t i = t; i >= b; --i) {
        phi *= -l[i + 1];
        psiB[i] = phi;
    }
}

// -----------------------------------------------------------------------------------------
// Solves along index i of a strided array (element i of column c at c*sc + i*si), real or
// complex: MODE 0, y = T^-1 x (forward L, diagonal, backward L^T); MODE 1, y = D^-1/2 L^-1 x,
// i.e. the rows b F^-1 with F = D^1/2 L^T (F^T F = T).  Helpers for both element types.
// -----------------------------------------------------------------------------------------
__device__ __forceinline__ double axmy(double x, double a, double y) { return fma(-a, y, x); }
__device__ __forceinline__ cplx axmy(cplx x, double a, cplx y) { return cmk(fma(-a, y.x, x.x), fma(-a, y.y, x.y)); }
__device__ __forceinline__ double sc_mul(double x, double s) { return x * s; }
__device__ __forceinline__ cplx sc_mul(cplx x, double s) { return cmk(x.x * s, x.y * s); }
__device__ __forceinline__ double maybe_conj(double x, int) { return x; }
__device__ __forceinline__ cplx maybe_conj(cplx x, int c) { return c ? cmk(x.x, -x.y) : x; }
__device__ __forceinline__ double fma_acc(double acc, double a, double x) { return fma(a, x, acc); }
__device__ __forceinline__ cplx fma_acc(cplx acc, double a, cplx x) { return cmk(fma(a, x.x, acc.x), fma(a, x.y, acc.y)); }
__device__ __forceinline__ double tsub(double a, double b) { return a - b; }
__device__ __forceinline__ double tadd(double a, double b) { return a + b; }
__device__ __forceinline__ cplx tadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx tsub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <> __device__ __forceinline__ cplx zero_of<cplx>() { return cmk(0, 0); }

// -----------------------------------------------------------------------------------------
// Chunked solves (MODE 0, T^-1 x; MODE 1, D^-1/2 L^-1 x): the recurrences split into chunks of
// CYC_CL steps solved from a zero start in parallel (one thread per chunk and column), a
// sequential pass per column over the chunks that carries the boundary values, and an
// elementwise pass that adds each chunk's propagator times its incoming value.  Exact in exact
// arithmetic (the superposition of a linear recurrence); the FP64 work spreads over the whole
// GPU instead of one lane per column.  part: 2 nch ncols + 2 nch ncols + ncols elements.
// -----------------------------------------------------------------------------------------
template <typename T>
__global__ void k_cyc_fwd_local(const T* in, T* out, int64_t N, int64_t ncols, int64_t si, int64_t sc,
                                const double* __restrict__ fac, T* part) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t col = tid % ncols, c = tid / ncols;
    if (c >= cyc_nch(N)) return;
    const double* l = fac;
    const double* m = fac + 2 * N;
    const T* x = in + col * sc;
    T* y = out + col * sc;
    T u = zero_of<T>(), acc = zero_of<T>();
    const int64_t s = 1 + c * CYC_CL, e = min(N - 1, s + CYC_CL);
    // groups of CYC_PF elements loaded before any is computed (the chain's loads would
    // otherwise wait one by one behind the stores, x and y possibly being the same array)
    for (int64_t i0 = s; i0 < e; i0 += CYC_PF) {
        T xv[CYC_PF];
        double lv[CYC_PF], mv[CYC_PF];
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t i = i0 + j;
            if (i < e) { xv[j] = x[i * si]; lv[j] = __ldg(l + i); mv[j] = __ldg(m + i); }
        }
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t i = i0 + j;
            if (i < e) {
                u = axmy(xv[j], lv[j], u);
                acc = fma_acc(acc, mv[j], u);
                y[i * si] = u;
            }
        }
    }
    part[2 * (c * ncols + col)] = u;
    part[2 * (c * ncols + col) + 1] = acc;
}

// per column: carry[c] = u_{s_c - 1}; tail = sum_{i <= N-2} m_i u_i
template <typename T>
__global__ void k_cyc_fwd_carry(const T* in, int64_t N, int64_t ncols, int64_t sc, const double* __restrict__ fac,
                                const T* part, T* carry, T* tail) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const double* m = fac + 2 * N;
    const double* psiF = fac + 4 * N;
    const double* msum = fac + 6 * N;
    const int64_t nch = cyc_nch(N);
    T cur = in[col * sc];                              // u_0 = x_0
    T s = zero_of<T>();
    s = fma_acc(s, m[0], cur);
    for (int64_t c0 = 0; c0 < nch; c0 += CYC_PF) {      // each group's loads issued together
        T pu[CYC_PF], ps[CYC_PF];
        double mv[CYC_PF], pe[CYC_PF];
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t c = c0 + j;
            if (c < nch) {
                pu[j] = part[2 * (c * ncols + col)];
                ps[j] = part[2 * (c * ncols + col) + 1];
                mv[j] = msum[c];
                pe[j] = psiF[min(N - 1, 1 + (c + 1) * CYC_CL) - 1];
            }
        }
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t c = c0 + j;
            if (c < nch) {
                carry[c * ncols + col] = cur;
                s = fma_acc(tadd(s, ps[j]), mv[j], cur);
                cur = fma_acc(pu[j], pe[j], cur);
            }
        }
    }
    tail[col] = s;
}

template <typename T, int MODE>
__global__ void k_cyc_fwd_fix(const T* in, T* out, int64_t N, int64_t ncols, int64_t si, int64_t sc,
                              const double* __restrict__ fac, const T* carry, const T* tail, int conj_out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * ncols) return;
    const int64_t col = idx % ncols, i = idx / ncols;
    const double* dinv = fac + N;
    const double* sd = fac + 3 * N;
    const double* psiF = fac + 4 * N;
    T u;
    if (i == 0) u = in[col * sc];
    else if (i == N - 1) u = tsub(in[col * sc + (N - 1) * si], tail[col]);
    else u = fma_acc(out[col * sc + i * si], psiF[i], carry[((i - 1) / CYC_CL) * ncols + col]);
    out[col * sc + i * si] = (MODE == 0) ? sc_mul(u, dinv[i]) : maybe_conj(sc_mul(u, sd[i]), conj_out);
}

// backward on w (in place): v_{N-2} = w_{N-2} - m_{N-2} w_{N-1}, v_i = (w_i - m_i w_{N-1}) - l_{i+1} v_{i+1}
template <typename T>
__global__ void k_cyc_bwd_local(T* y, int64_t N, int64_t ncols, int64_t si, int64_t sc, const double* __restrict__ fac,
                                T* part) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t col = tid % ncols, c = tid / ncols;
    if (c >= cyc_nch(N)) return;
    const double* l = fac;
    const double* m = fac + 2 * N;
    T* yc = y + col * sc;
    const T yl = yc[(N - 1) * si];
    T v = zero_of<T>();
    const int64_t t = N - 3 - c * CYC_CL, b = max((int64_t)0, t - CYC_CL + 1);
    for (int64_t i0 = t; i0 >= b; i0 -= CYC_PF) {
        T wv[CYC_PF];
        double lv[CYC_PF], mv[CYC_PF];
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t i = i0 - j;
            if (i >= b) { wv[j] = yc[i * si]; lv[j] = __ldg(l + i + 1); mv[j] = __ldg(m + i); }
        }
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t i = i0 - j;
            if (i >= b) {
                v = axmy(axmy(wv[j], mv[j], yl), lv[j], v);
                yc[i * si] = v;
            }
        }
    }
    part[c * ncols + col] = v;
}

template <typename T>
__global__ void k_cyc_bwd_carry(const T* y, int64_t N, int64_t ncols, int64_t si, int64_t sc,
                                const double* __restrict__ fac, const T* part, T* carry) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const double* m = fac + 2 * N;
    const double* psiB = fac + 5 * N;
    const T* yc = y + col * sc;
    T cur = axmy(yc[(N - 2) * si], m[N - 2], yc[(N - 1) * si]);     // v_{N-2}
    const int64_t nch = cyc_nch(N);
    for (int64_t c0 = 0; c0 < nch; c0 += CYC_PF) {
        T pv[CYC_PF];
        double pb[CYC_PF];
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t c = c0 + j;
            if (c < nch) {
                pv[j] = part[c * ncols + col];
                pb[j] = psiB[max((int64_t)0, N - 3 - c * CYC_CL - CYC_CL + 1)];
            }
        }
#pragma unroll
        for (int j = 0; j < CYC_PF; ++j) {
            const int64_t c = c0 + j;
            if (c < nch) {
                carry[c * ncols + col] = cur;
                cur = fma_acc(pv[j], pb[j], cur);
            }
        }
    }
}

template <typename T>
__global__ void k_cyc_bwd_fix(T* y, int64_t N, int64_t ncols, int64_t si, int64_t sc, const double* __restrict__ fac,
                              const T* carry, int conj_out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * ncols) return;
    const int64_t col = idx % ncols, i = idx / ncols;
    const double* m = fac + 2 * N;
    const double* psiB = fac + 5 * N;
    T* yc = y + col * sc;
    T v;
    if (i == N - 1) v = yc[i * si];
    else if (i == N - 2) v = axmy(yc[i * si], m[N - 2], yc[(N - 1) * si]);
    else v = fma_acc(yc[i * si], psiB[i], carry[((N - 3 - i) / CYC_CL) * ncols + col]);
    // every thread of column col reads y[N-1], y[N-2] above; they are rewritten only by
    // their own threads with values derived from themselves in an earlier pass, so the
    // final values are written in a separate launch (k_cyc_bwd_ends) to keep reads race-free
    if (i < N - 2) yc[i * si] = maybe_conj(v, conj_out);
}

template <typename T>
__global__ void k_cyc_bwd_ends(T* y, int64_t N, int64_t ncols, int64_t si, int64_t sc, const double* __restrict__ fac,
                               int conj_out) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const double* m = fac + 2 * N;
    T* yc = y + col * sc;
    const T yl = yc[(N - 1) * si];
    yc[(N - 2) * si] = maybe_conj(axmy(yc[(N - 2) * si], m[N - 2], yl), conj_out);
    yc[(N - 1) * si] = maybe_conj(yl, conj_out);
}

// tridiagonal coefficients of G (cL = 0, cG = 1) or L (cL = 1, cG = 0): ab[i] = T_ii,
// ab[N + i] = T_{i,i+1}
__global__ void k_tri_ab(const double* __restrict__ h, int N, double cL, double cG, double* ab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    ab[i] = tri_diag(h, N, i, cL, cG);
    ab[N + i] = tri_off(h, i, cL, cG);
}

// y = T x, T from its coefficients ab, on the columns of a real N x ncols block, column-major
// (element (i, c) at c N + i) or row-major (at i ncols + c)
template <bool ROWMAJOR>
__global__ void k_tri_mul(const double* __restrict__ x, double* __restrict__ y, int64_t N, int64_t ncols,
                          const double* __restrict__ ab) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * ncols) return;
    const int64_t i = ROWMAJOR ? idx / ncols : idx % N;
    const int64_t c = ROWMAJOR ? idx % ncols : idx / N;
    const int64_t ip = (i == 0) ? N - 1 : i - 1, in = (i == N - 1) ? 0 : i + 1;
    const int64_t si = ROWMAJOR ? ncols : 1, base = ROWMAJOR ? c : c * N;
    double v = __ldg(ab + i) * x[base + i * si];
    v = fma(__ldg(ab + N + ip), x[base + ip * si], v);
    v = fma(__ldg(ab + N + i), x[base + in * si], v);
    y[idx] = v;
}

// Chebyshev step on equal-layout blocks: out = a Z + c Yc - Yp (Yp may be null)
__global__ void k_cheb_comb(double* __restrict__ out, const double* __restrict__ Z, const double* __restrict__ Yc,
                            const double* __restrict__ Yp, int64_t cnt, double a, double c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    double v = fma(a, Z[i], c * Yc[i]);
    if (Yp) v -= Yp[i];
    out[i] = v;
}

// s[i] = sum_{e < i} h_e (arclength at vertex i), s[N] = perimeter; one thread, fixed order
__global__ void k_arclength(const double* __restrict__ h, int N, double* s) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double a = 0.0;
    for (int i = 0; i < N; ++i) { s[i] = a; a += h[i]; }
    s[N] = a;
}

// Starting basis of the subspace iteration: arclength Fourier modes, column c of X (N x p,
// row-major): 1, cos(2 pi m s_i / P), sin(2 pi m s_i / P) for m = 1, 2, ... (cos and sin adjacent)
__global__ void k_fourier_arc(double* X, int64_t N, int64_t p, const double* __restrict__ s) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * p) return;
    const int64_t i = idx / p;
    const int c = (int)(idx % p);
    double v = 1.0;
    if (c > 0) {
        const int m = (c + 1) / 2;
        double t = (double)m * (s[i] / s[N]);
        t -= floor(t);
        double sn, cs;
        sincospi(2.0 * t, &sn, &cs);
        v = (c & 1) ? cs : sn;
    }
    X[idx] = v;
}

// -----------------------------------------------------------------------------------------
// Real GEMM C = op(A) op(B) (column-major, FP64 in and out) in double-float on the FP32 pipe:
// GB300 issues FP32 at 64x its FP64 rate, and in FP64 these products ran at the FP64 roofline.
// 64 x 64 tiles, 16-deep K slices staged in shared memory as hi + lo float pairs (split from
// the bit fields with integer operations: the FP64 pipe's conversions took a third of its
// cycles; operands below 2^-74 in magnitude, far below the basis' entries, stage as zero),
// 4 x 4 outputs per thread, Dekker products and two-sum accumulation, results rounded to double.
// About 48 significant bits per operation, so a K-term sum carries errors of order
// sqrt(K) 2^-48 of its terms' magnitudes.  Split K: blockIdx.z takes K indices
// [z kchunk, (z + 1) kchunk) and writes its partial product to C + z zstride.
// -----------------------------------------------------------------------------------------
// TRI: op(A) is lower triangular (A[k, m] = 0 for k > m, an upper-triangular A taken
// transposed), so a tile of rows m0.. needs K only below m0 + 64.
template <int OPA, int OPB, bool TRI>
__global__ void __launch_bounds__(256) k_dgemm_df(int M, int Nc, int K, const double* __restrict__ A, int64_t lda,
                                                  const double* __restrict__ B, int64_t ldb, double* C, int64_t ldc,
                                                  int kchunk, int64_t zstride) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN + 1];
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * kchunk, ke = min(min(K, kb + kchunk), TRI ? m0 + BM : K);
    C += blockIdx.z * zstride;
    dfl acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = {0.f, 0.f};
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int mm, kk;
            if (OPA == OP_N) { mm = t % 64; kk = t / 64 + 4 * s; } else { kk = t % 16; mm = t / 16 + 16 * s; }
            const int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < ke) v = (OPA == OP_N) ? A[gm + (int64_t)gk * lda] : A[gk + (int64_t)gm * lda];
            const dfl d = dfl_from_bits(v);
            As[kk][mm] = make_float2(d.hi, d.lo);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int kk, nn;
            if (OPB == OP_N) { kk = t % 16; nn = t / 16 + 16 * s; } else { nn = t % 64; kk = t / 64 + 4 * s; }
            const int gk = k0 + kk, gn = n0 + nn;
            double v = 0.0;
            if (gk < ke && gn < Nc) v = (OPB == OP_N) ? B[gk + (int64_t)gn * ldb] : B[gn + (int64_t)gk * ldb];
            const dfl d = dfl_from_bits(v);
            Bs[kk][nn] = make_float2(d.hi, d.lo);
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < BK; ++kk) {
            dfl a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = dfl_mk(As[kk][tx + 16 * i]);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = dfl_mk(Bs[kk][ty + 16 * j]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = dfl_fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tx + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + ty + 16 * j;
            if (gn >= Nc) continue;
            C[gm + (int64_t)gn * ldc] = dfl_to(acc[i][j]);
        }
    }
}

// C = sum over z of P[z] (fixed order), count entries each
__global__ void k_sum_splits(const double* __restrict__ P, int nz, int64_t count, double* C) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double v = P[i];
    for (int z = 1; z < nz; ++z) v += P[z * count + i];
    C[i] = v;
}

// -----------------------------------------------------------------------------------------
// One CTA: upper Cholesky factor of a small SPD matrix, C + shift I = R^T R (C column-major,
// ld p), in double-float on the FP32 pipe, blocked by panels of CHOL_NB rows: the upper
// triangle is copied into W (p^2 float pairs); each panel (its rows of the upper triangle)
// is staged in shared memory and factored there, written back, and the trailing triangle
// receives one rank-CHOL_NB update per panel, reading the panel from shared memory (the
// unblocked form streamed the trailing triangle through the SM at every pivot).  R is then
// written back to C's upper triangle and mirrored into its strict lower triangle
// (C[k + i p] = R_ik, where a row of R is contiguous); when Rc is given, R is also copied as
// complex (strict lower part zero: the input of the Jacobi SVD).  Pivot square roots and
// reciprocals: one Newton correction of the FP32 values, r = s + (v - s^2)/(2 s) and
// q + q (1 - q r).  A pivot that is not positive sets DEVERR_SINGULAR (and is replaced by 1
// so the kernel ends).  Dynamic shared memory: chol_smem_bytes(p).
// -----------------------------------------------------------------------------------------
#define CHOL_NB 16
static size_t chol_smem_bytes(int p) { return sizeof(float2) * CHOL_NB * (size_t)p; }

__global__ void __launch_bounds__(1024) k_chol(double* C, float2* W, int p, double shift, cplx* Rc, double* rdiag,
                                               int* err) {
    extern __shared__ float2 pan[];        // CHOL_NB rows x p columns (row r at pan + r p)
    __shared__ float2 s_ir;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t idx = tid; idx < (int64_t)p * p; idx += nt) {
        const int i = (int)(idx % p), k = (int)(idx / p);
        if (i <= k) {
            const dfl d = dfl_from(C[idx] + (i == k ? shift : 0.0));
            W[idx] = make_float2(d.hi, d.lo);
        }
    }
    __syncthreads();
    for (int jb = 0; jb < p; jb += CHOL_NB) {
        const int nb = min(CHOL_NB, p - jb);
        for (int idx = tid; idx < nb * p; idx += nt) {
            const int r = idx / p, k = idx % p;
            if (k >= jb + r) pan[r * p + k] = W[(jb + r) + (int64_t)k * p];
        }
        __syncthreads();
        for (int jj = 0; jj < nb; ++jj) {
            const int j = jb + jj;
            if (tid == 0) {
                dfl v = dfl_mk(pan[jj * p + j]);
                if (!(v.hi > 0.0f)) { atomicOr(err, DEVERR_SINGULAR); v = {1.0f, 0.0f}; }
                const float sr = sqrtf(v.hi);
                const float res = fmaf(-sr, sr, v.hi) + v.lo;
                const dfl r = dfl_qts(sr, res / (2.0f * sr));
                const float q = 1.0f / r.hi;
                const float e = fmaf(-q, r.hi, 1.0f) - q * r.lo;
                const dfl ir = dfl_qts(q, q * e);
                pan[jj * p + j] = make_float2(r.hi, r.lo);
                s_ir = make_float2(ir.hi, ir.lo);
                if (rdiag) rdiag[j] = dfl_to(ir);
            }
            __syncthreads();
            const dfl ir = dfl_mk(s_ir);
            for (int k = j + 1 + tid; k < p; k += nt) {
                const dfl v = dfl_mul(dfl_mk(pan[jj * p + k]), ir);
                pan[jj * p + k] = make_float2(v.hi, v.lo);
            }
            __syncthreads();
            // the panel's later rows: pan[rr][k] -= R_{j, jb+rr} R_{j, k}  (k >= jb + rr)
            const int nr = nb - jj - 1, nk = p - j - 1;
            for (int idx = tid; idx < nr * nk; idx += nt) {
                const int rr = jj + 1 + idx / nk, k = j + 1 + idx % nk;
                if (k >= jb + rr) {
                    const float2 a = pan[jj * p + jb + rr];
                    const dfl w = dfl_fma(dfl_mk(make_float2(-a.x, -a.y)), dfl_mk(pan[jj * p + k]), dfl_mk(pan[rr * p + k]));
                    pan[rr * p + k] = make_float2(w.hi, w.lo);
                }
            }
            __syncthreads();
        }
        for (int idx = tid; idx < nb * p; idx += nt) {
            const int r = idx / p, k = idx % p;
            if (k >= jb + r) W[(jb + r) + (int64_t)k * p] = pan[r * p + k];
        }
        // trailing triangle: W_ik -= sum_r R_{jb+r, i} R_{jb+r, k}  (jb + nb <= i <= k)
        const int t0 = jb + nb, m = p - t0;
        for (int64_t idx = tid; idx < (int64_t)m * m; idx += nt) {
            const int i = t0 + (int)(idx % m), k = t0 + (int)(idx / m);
            if (i > k) continue;
            dfl acc = {0.f, 0.f};
            for (int r = 0; r < nb; ++r) acc = dfl_fma(dfl_mk(pan[r * p + i]), dfl_mk(pan[r * p + k]), acc);
            const dfl w = dfl_sub(dfl_mk(W[i + (int64_t)k * p]), acc);
            W[i + (int64_t)k * p] = make_float2(w.hi, w.lo);
        }
        __syncthreads();
    }
    for (int64_t idx = tid; idx < (int64_t)p * p; idx += nt) {
        const int i = (int)(idx % p), k = (int)(idx / p);
        if (i <= k) {
            const double v = dfl_to(dfl_mk(W[idx]));
            C[idx] = v;
            if (i < k) C[k + (int64_t)i * p] = v;        // R_ik into the lower triangle
        }
        if (Rc) Rc[idx] = cmk(i <= k ? dfl_to(dfl_mk(W[idx])) : 0.0, 0.0);
    }
}

// Rinv = R^-1 (upper, ld p; strict lower part zero) from the mirrored factor of k_chol and the
// pivots' reciprocals rdiag: one warp per column, x_i = -(sum_{k=i+1..j} R_ik x_k) / R_ii, the
// sum over the lanes (R_ik at C[k + i p], contiguous in k) reduced in a fixed order
__global__ void __launch_bounds__(256) k_tri_inv(const double* __restrict__ C, const double* __restrict__ rdiag, int p,
                                                 double* Rinv) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= p) return;
    double* x = Rinv + (int64_t)j * p;
    for (int i = j + 1 + lane; i < p; i += 32) x[i] = 0.0;
    if (lane == 0) x[j] = rdiag[j];
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
        const double* ri = C + (int64_t)i * p;
        double acc = 0.0;
        for (int k = i + 1 + lane; k <= j; k += 32) acc = fma(ri[k], x[k], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] = -acc * rdiag[i];
        __syncwarp();
    }
}

// Cf[:, c] = Re E[:, first + c] (p x nc, ld p) and gm[c] = 1
__global__ void k_take_cols(const cplx* __restrict__ E, int p, int first, int nc, double* Cf, double* gm) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)p * nc) return;
    const int i = (int)(idx % p), c = (int)(idx / p);
    Cf[idx] = E[i + (int64_t)(first + c) * p].x;
    if (i == 0) gm[c] = 1.0;
}

__global__ void k_iota(int* v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

// =========================================================================================
// Host side
// =========================================================================================
namespace {
// consecutive 256-byte-aligned parts of the handle's workspace
struct WorkParts {
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> parts;
    void add(void** p, size_t bytes) { parts.push_back({p, bytes}); off += (bytes + 255) & ~size_t(255); }
    bem_status commit(bem_ctx* h) {
        void* base = nullptr;
        bem_status st = bem_workspace(h, off, &base);
        if (st != BEM_OK) return st;
        size_t o = 0;
        for (auto& pr : parts) { *pr.first = (char*)base + o; o += (pr.second + 255) & ~size_t(255); }
        return BEM_OK;
    }
};
}  // namespace

bem_status launch_cyc_factor(bem_ctx* h, double cL, double cG, double* fac) {
    const int N = (int)h->N;
    const unsigned g = (unsigned)((N + 255) / 256);
    const unsigned gc = (unsigned)((cyc_nch(N) + 127) / 128), gf = (unsigned)((fac_nch(N) + 127) / 128);
    const int64_t N64 = N;
    BEM_TIMED(h, "k_cyc_factor", (k_tri_coef<<<g, 256, 0, h->stream>>>(h->seg + 4 * h->N, N, cL, cG, fac),
                                  k_fac_transfer<<<gf, 128, 0, h->stream>>>(N64, fac),
                                  k_fac_carry<<<1, 1, 0, h->stream>>>(N64, fac),
                                  k_fac_pivots<<<gf, 128, 0, h->stream>>>(N64, fac, h->dev_err),
                                  k_fac_border_carry<<<1, 1, 0, h->stream>>>(N64, fac),
                                  k_fac_border<<<gf, 128, 0, h->stream>>>(N64, fac),
                                  k_fac_final<<<1, 1, 0, h->stream>>>(N64, fac, h->dev_err),
                                  k_cyc_prop<<<gc, 128, 0, h->stream>>>(N64, fac)));
    BEM_LAUNCH(h, "k_cyc_factor");
    return BEM_OK;
}

size_t cyc_factor_bytes(int64_t N) { return sizeof(double) * CYC_FAC * (size_t)N; }
template <typename T>
static size_t cyc_scratch_elems(int64_t N, int64_t ncols) { return (size_t)(5 * cyc_nch(N) * ncols + ncols); }

// the chunked solve of mode 0 (T^-1) or 1 (D^-1/2 L^-1) on h's stream; scratch: at least
// cyc_scratch_elems elements of T
template <typename T>
static bem_status cyc_solve_chunked(bem_ctx* h, int mode, const T* in, T* out, int64_t N, int64_t ncols, int64_t si,
                                    int64_t sc, const double* fac, T* scratch, bool conj_out) {
    const int64_t nch = cyc_nch(N);
    T* partF = scratch;                     // 2 nch ncols
    T* carryF = partF + 2 * nch * ncols;    // nch ncols
    T* partB = carryF + nch * ncols;        // nch ncols
    T* carryB = partB + nch * ncols;        // nch ncols
    T* tail = carryB + nch * ncols;         // ncols
    const unsigned gl = (unsigned)((nch * ncols + 127) / 128), gcol = (unsigned)((ncols + 127) / 128),
                   gall = (unsigned)((N * ncols + 255) / 256);
    const int cj = conj_out ? 1 : 0;
    BEM_TIMED(h, "k_cyc_solve",
              (k_cyc_fwd_local<T><<<gl, 128, 0, h->stream>>>(in, out, N, ncols, si, sc, fac, partF),
               k_cyc_fwd_carry<T><<<gcol, 128, 0, h->stream>>>(in, N, ncols, sc, fac, partF, carryF, tail)));
    if (mode == 1) {
        BEM_TIMED(h, "k_cyc_solve", (k_cyc_fwd_fix<T, 1><<<gall, 256, 0, h->stream>>>(in, out, N, ncols, si, sc, fac, carryF,
                                                                                       tail, cj)));
        BEM_LAUNCH(h, "k_cyc_solve");
        return BEM_OK;
    }
    BEM_TIMED(h, "k_cyc_solve",
              (k_cyc_fwd_fix<T, 0><<<gall, 256, 0, h->stream>>>(in, out, N, ncols, si, sc, fac, carryF, tail, 0),
               k_cyc_bwd_local<T><<<gl, 128, 0, h->stream>>>(out, N, ncols, si, sc, fac, partB),
               k_cyc_bwd_carry<T><<<gcol, 128, 0, h->stream>>>(out, N, ncols, si, sc, fac, partB, carryB),
               k_cyc_bwd_fix<T><<<gall, 256, 0, h->stream>>>(out, N, ncols, si, sc, fac, carryB, cj),
               k_cyc_bwd_ends<T><<<gcol, 128, 0, h->stream>>>(out, N, ncols, si, sc, fac, cj)));
    BEM_LAUNCH(h, "k_cyc_solve");
    return BEM_OK;
}

bem_status general_gram_apply(bem_ctx* h, int mode, const cplx* in, cplx* out, cplx* tmp, size_t tmp_elems, int64_t N,
                              int64_t ncols, int64_t si, int64_t sc, bool conj_out) {
    if (!h->gfac) return bem_fail(h, BEM_E_INVALID, "Gram solve: no factor of the general Gram matrix");
    if (!tmp || tmp_elems < cyc_scratch_elems<cplx>(N, ncols))
        return bem_fail(h, BEM_E_INVALID, "Gram solve: the general mesh's chunked solve needs scratch");
    return cyc_solve_chunked<cplx>(h, mode, in, out, N, ncols, si, sc, h->gfac, tmp, conj_out);
}

template <int OPA, int OPB, bool TRI = false>
static bem_status dgemm_t(bem_ctx* h, int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B,
                          int64_t ldb, double* C, int64_t ldc, int nz = 1, int kchunk = 0, int64_t zstride = 0) {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((Nc + 63) / 64), (unsigned)nz);
    BEM_TIMED(h, TRI ? "k_dgemm_df_tri" : "k_dgemm_df",
              (k_dgemm_df<OPA, OPB, TRI><<<grid, 256, 0, h->stream>>>((int)M, (int)Nc, (int)K, A, lda, B,
                                                                                         ldb, C, ldc,
                                                                                         nz == 1 ? (int)K : kchunk, zstride)));
    BEM_LAUNCH(h, "k_dgemm_df");
    return BEM_OK;
}

// splits of the long-K Gram products (p x p over K = N): enough CTAs for two waves
static int gram_splits(int64_t p, int64_t K) {
    const int64_t tiles = ((p + 63) / 64) * ((p + 63) / 64);
    int64_t z = (2 * 152 + tiles - 1) / tiles;
    z = std::min<int64_t>(z, std::max<int64_t>(1, K / 256));
    return (int)std::max<int64_t>(1, std::min<int64_t>(z, 64));
}

// C = X^T Z (p x p, ld p) for row-major N x p blocks X, Z (column-major p x N, ld p), split
// over N into `part` (gram_splits(p, N) p^2 doubles) and summed in a fixed order
static bem_status gram_product(bem_ctx* h, int64_t p, int64_t N, const double* X, const double* Z, double* C, double* part) {
    const int nz = gram_splits(p, N);
    int kchunk = (int)((N + nz - 1) / nz);
    kchunk = (kchunk + 15) & ~15;
    bem_status st = dgemm_t<OP_N, OP_T>(h, p, p, N, X, p, Z, p, part, p, nz, kchunk, p * p);
    if (st != BEM_OK) return st;
    BEM_TIMED(h, "k_sum_splits", (k_sum_splits<<<(unsigned)((p * p + 255) / 256), 256, 0, h->stream>>>(part, nz, p * p, C)));
    BEM_LAUNCH(h, "k_sum_splits");
    return BEM_OK;
}

static bem_status tri_mul(bem_ctx* h, const double* x, double* y, int64_t ncols, const double* ab, bool rowmajor) {
    const int64_t tot = h->N * ncols;
    const unsigned g = (unsigned)((tot + 255) / 256);
    if (rowmajor) {
        BEM_TIMED(h, "k_tri_mul", (k_tri_mul<true><<<g, 256, 0, h->stream>>>(x, y, h->N, ncols, ab)));
    } else {
        BEM_TIMED(h, "k_tri_mul", (k_tri_mul<false><<<g, 256, 0, h->stream>>>(x, y, h->N, ncols, ab)));
    }
    BEM_LAUNCH(h, "k_tri_mul");
    return BEM_OK;
}

// W: p^2 float2 scratch of the factorisation; rdiag (p doubles, or null) receives 1/R_jj
static bem_status chol_launch(bem_ctx* h, double* C, float2* W, int64_t p, double shift, cplx* Rc, double* rdiag) {
    const size_t sm = chol_smem_bytes((int)p);
    BEM_CUDA(h, cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    BEM_TIMED(h, "k_chol", (k_chol<<<1, 1024, sm, h->stream>>>(C, W, (int)p, shift, Rc, rdiag, h->dev_err)));
    BEM_LAUNCH(h, "k_chol");
    return BEM_OK;
}

static bem_status chol_inv(bem_ctx* h, double* C, float2* W, double* rdiag, int64_t p, double* Rinv) {
    bem_status st = chol_launch(h, C, W, p, 0.0, nullptr, rdiag);
    if (st != BEM_OK) return st;
    BEM_TIMED(h, "k_tri_inv", (k_tri_inv<<<(unsigned)((p + 7) / 8), 256, 0, h->stream>>>(C, rdiag, (int)p, Rinv)));
    BEM_LAUNCH(h, "k_tri_inv");
    return BEM_OK;
}

// block size of the subspace iteration for n wanted pairs, and its iteration count
void general_basis_plan(int64_t N, int64_t n, double perimeter, int64_t* p_out, int* iters_out, double* sigma_out,
                        double* bound_out) {
    // block: measured at N = 16384, n = 201 against 2n + 9 and 1.75 n + 9 (the one-CTA
    // Cholesky and the Jacobi grow as p^3, the products as N p^2, the step count as the
    // separation below shrinks)
    int64_t p = n + n / 2 + 9;
    if (p > 1023) p = 1023;
    if (p > N - 1) p = N - 1;
    if (p < n) p = n;
    // The operator sigma (L + sigma G)^-1 G has the eigenvalues mu = sigma / (lambda + sigma).
    // The pencil's eigenvalues bound those of the curve's Laplace-Beltrami operator,
    // lambda = (2 pi m / P)^2 on the polygon's perimeter P, from above (conforming P1
    // Galerkin), so every unwanted mu lies in [0, b], b = sigma / (lambda_{p+1} + sigma): the
    // interval the Chebyshev steps damp.  Degree: T_d(2 mu_n / b - 1) >= 1e17 on the wanted
    // end, plus two.
    const double w = 2.0 * BEM_PI / perimeter;
    const double mn = (double)((n - 1) / 2 + 1), mp = (double)((p + 1) / 2);
    const double lam_n = (w * mn) * (w * mn), lam_p = (w * mp) * (w * mp);
    const double sigma = std::max(0.25 * lam_n, w * w);
    const double mu_n = sigma / (lam_n + sigma), b = sigma / (lam_p + sigma);
    const double x0 = 2.0 * mu_n / b - 1.0;
    int it = (x0 > 1.0) ? (int)ceil(acosh(1e17) / acosh(x0)) + 2 : 400;
    *p_out = p;
    *iters_out = std::min(std::max(it, 3), 400);
    *sigma_out = sigma;
    *bound_out = b;
}

static bem_status read_basis_err(bem_ctx* h) {
    int e = 0;
    BEM_CUDA(h, cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (e) {
        BEM_CUDA(h, cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
        if (e & DEVERR_TIMEOUT) return bem_fail(h, BEM_E_TIMEOUT, "filter basis: a device-side wait timed out");
        return bem_fail(h, BEM_E_SINGULAR, "filter basis: a Cholesky pivot of the subspace iteration is not positive");
    }
    return BEM_OK;
}

// The filter basis of a non-equal-chord mesh: h->Q (N x nc, G-orthonormal) spans the
// eigenvectors of the nc lowest eigenvalues of L phi = lambda G phi (without the constant
// mode when inc = 0), h->GQ = G h->Q and h->gm = 1 (the basis is G-orthonormal, so the
// diagonal Gram scaling of the equal-chord path is the identity here).
bem_status general_filter_basis(bem_ctx* h, int64_t nc, int inc) {
    const int64_t N = h->N;
    const int64_t n = inc ? nc : nc + 1;
    int64_t p;
    int iters;
    double sigma, bnd;
    general_basis_plan(N, n, h->hbar * (double)N, &p, &iters, &sigma, &bnd);
    h->basis_block = (int)p;
    h->basis_iters = iters;
    double *X = nullptr, *Y = nullptr, *Z = nullptr, *Wb = nullptr, *Vb = nullptr, *C = nullptr, *Rinv = nullptr,
           *Cf = nullptr, *fac = nullptr,
           *s = nullptr, *sig = nullptr, *part = nullptr, *abG = nullptr, *abL = nullptr, *abGs = nullptr,
           *cscr = nullptr, *rdg = nullptr;
    cplx *Rc = nullptr, *E = nullptr;
    float2* Wdf = nullptr;
    int* perm = nullptr;
    void* jac = nullptr;
    WorkParts cv;
    cv.add((void**)&X, sizeof(double) * N * p);
    cv.add((void**)&Y, sizeof(double) * N * p);
    cv.add((void**)&Z, sizeof(double) * N * p);
    cv.add((void**)&Wb, sizeof(double) * N * p);
    cv.add((void**)&Vb, sizeof(double) * N * p);
    cv.add((void**)&C, sizeof(double) * p * p);
    cv.add((void**)&Rinv, sizeof(double) * p * p);
    cv.add((void**)&Wdf, sizeof(float2) * p * p);
    cv.add((void**)&rdg, sizeof(double) * p);
    cv.add((void**)&part, sizeof(double) * p * p * gram_splits(p, N));
    cv.add((void**)&Cf, sizeof(double) * p * nc);
    cv.add((void**)&fac, cyc_factor_bytes(N));
    cv.add((void**)&cscr, sizeof(double) * cyc_scratch_elems<double>(N, p));
    cv.add((void**)&abG, sizeof(double) * 2 * N);
    cv.add((void**)&abL, sizeof(double) * 2 * N);
    cv.add((void**)&abGs, sizeof(double) * 2 * N);
    cv.add((void**)&s, sizeof(double) * (N + 1));
    cv.add((void**)&sig, sizeof(double) * p);
    cv.add((void**)&Rc, sizeof(cplx) * p * p);
    cv.add((void**)&E, sizeof(cplx) * p * p);
    cv.add((void**)&perm, sizeof(int) * p);
    cv.add(&jac, jacobi_scratch_bytes((int)p));
    bem_status st;
    if ((st = cv.commit(h)) != BEM_OK) return st;
    // (L + sigma G) = L D L^T for the shift-and-invert steps; the coefficients of G and L
    if ((st = launch_cyc_factor(h, 1.0, sigma, fac)) != BEM_OK) return st;
    const unsigned gN = (unsigned)((N + 255) / 256);
    // the steps apply sigma (L + sigma G)^-1 G, whose eigenvalues sigma / (lambda + sigma) lie in
    // (0, 1]: the iterates never grow, whatever the curve's size (the double-float products
    // stage floats)
    BEM_TIMED(h, "k_tri_ab", (k_tri_ab<<<gN, 256, 0, h->stream>>>(h->seg + 4 * N, (int)N, 0.0, 1.0, abG),
                              k_tri_ab<<<gN, 256, 0, h->stream>>>(h->seg + 4 * N, (int)N, 1.0, 0.0, abL),
                              k_tri_ab<<<gN, 256, 0, h->stream>>>(h->seg + 4 * N, (int)N, 0.0, sigma, abGs)));
    BEM_LAUNCH(h, "k_tri_ab");
    BEM_TIMED(h, "k_arclength", (k_arclength<<<1, 1, 0, h->stream>>>(h->seg + 4 * N, (int)N, s)));
    BEM_LAUNCH(h, "k_arclength");
    BEM_TIMED(h, "k_fourier_arc", (k_fourier_arc<<<(unsigned)((N * p + 255) / 256), 256, 0, h->stream>>>(X, N, p, s)));
    BEM_LAUNCH(h, "k_fourier_arc");
    // The basis blocks X, Y, Z are row-major N x p, so the chunked solves' threads (adjacent
    // columns of one chunk) read adjacent addresses.  G-orthonormalise the columns of `in` into `out`:
    // R^T R = in^T G in, out = in R^-1 (as out^T = R^-T in^T)
    auto cholqr = [&](const double* in, double* out) -> bem_status {
        bem_status q;
        if ((q = tri_mul(h, in, Z, p, abG, true)) != BEM_OK) return q;
        if ((q = gram_product(h, p, N, in, Z, C, part)) != BEM_OK) return q;
        if ((q = chol_inv(h, C, Wdf, rdg, p, Rinv)) != BEM_OK) return q;
        return dgemm_t<OP_T, OP_N, true>(h, p, N, p, Rinv, p, in, p, out, p);     // R^-1 upper triangular
    };
    if ((st = cholqr(X, Y)) != BEM_OK) return st;
    std::swap(X, Y);
    // Chebyshev subspace iteration on the damped interval [0, b] of T = sigma (L + sigma G)^-1 G:
    // with S = (2/b) T - I, Y_0 = X, Y_1 = S Y_0, Y_{d+1} = 2 S Y_d - Y_{d-1}; the wanted
    // components grow as T_d(2 mu / b - 1) while every unwanted one stays within [-1, 1] (plain
    // powers of T needed 56 steps for n = 201 where this needs 24).  The pair (Y_d, Y_{d+1}) is
    // re-orthonormalised by one right factor (the recurrence is linear in the pair) every
    // second step and at each of the last two: a step widens the spread of the components by
    // at most T_1(2/b - 1) < 4/b (about 40 for p = 1.5 n), so the Gram matrix of the second
    // step stays far inside what the double-float Cholesky factors.
    const int64_t cnt = N * p;
    const unsigned gcm = (unsigned)((cnt + 255) / 256);
    auto apply_T = [&](const double* in, double* out) -> bem_status {    // out = T in
        bem_status q;
        if ((q = tri_mul(h, in, out, p, abGs, true)) != BEM_OK) return q;
        return cyc_solve_chunked<double>(h, 0, out, out, N, p, p, 1, fac, cscr, false);
    };
    auto comb = [&](double* out, const double* Zs, const double* Yc_, const double* Yp_, double a_, double c_) -> bem_status {
        BEM_TIMED(h, "k_cheb_comb", (k_cheb_comb<<<gcm, 256, 0, h->stream>>>(out, Zs, Yc_, Yp_, cnt, a_, c_)));
        BEM_LAUNCH(h, "k_cheb_comb");
        return BEM_OK;
    };
    double *Yp = X, *Yc = Y, *F1 = Wb, *F2 = Vb;
    if ((st = apply_T(Yp, Z)) != BEM_OK) return st;
    if ((st = comb(Yc, Z, Yp, nullptr, 2.0 / bnd, -1.0)) != BEM_OK) return st;
    for (int d = 1; d < iters; ++d) {
        if ((st = apply_T(Yc, Z)) != BEM_OK) return st;
        if ((st = comb(F1, Z, Yc, Yp, 4.0 / bnd, -2.0)) != BEM_OK) return st;      // Y_{d+1}
        if (d % 2 == 1 || d >= iters - 2) {
            if ((st = cholqr(F1, F2)) != BEM_OK) return st;                        // Y_{d+1} R^-1
            if ((st = dgemm_t<OP_T, OP_N, true>(h, p, N, p, Rinv, p, Yc, p, F1, p)) != BEM_OK) return st;   // Y_d R^-1
            double *oYp = Yp, *oYc = Yc;
            Yp = F1; Yc = F2; F1 = oYp; F2 = oYc;
        } else {
            double* oYp = Yp;
            Yp = Yc; Yc = F1; F1 = oYp;
        }
    }
    X = Yc;
    // Rayleigh-Ritz: A = X^T L X; the eigenvectors of A + sigma I are the right singular
    // vectors of its Cholesky factor (Jacobi SVD, sorted by decreasing singular value)
    if ((st = tri_mul(h, X, Z, p, abL, true)) != BEM_OK) return st;
    if ((st = gram_product(h, p, N, X, Z, C, part)) != BEM_OK) return st;
    if ((st = chol_launch(h, C, Wdf, p, sigma, Rc, nullptr)) != BEM_OK) return st;
    BEM_TIMED(h, "k_iota", (k_iota<<<(unsigned)((p + 255) / 256), 256, 0, h->stream>>>(perm, (int)p)));
    BEM_LAUNCH(h, "k_iota");
    if ((st = launch_jacobi_svd(h, Rc, (int)p, perm, sig, E, jac)) != BEM_OK) return st;
    // the n lowest Ritz vectors are the last n columns; without the kernel mode the very last
    // (the constant vector, lambda = 0) is left out
    BEM_TIMED(h, "k_take_cols", (k_take_cols<<<(unsigned)((p * nc + 255) / 256), 256, 0, h->stream>>>(E, (int)p, (int)(p - n),
                                                                                                   (int)nc, Cf, h->gm)));
    BEM_LAUNCH(h, "k_take_cols");
    // Q = X Cf (column-major N x nc)
    if ((st = dgemm_t<OP_T, OP_N>(h, N, nc, p, X, p, Cf, p, h->Q, N)) != BEM_OK) return st;
    if ((st = tri_mul(h, h->Q, h->GQ, nc, abG, false)) != BEM_OK) return st;
    return read_basis_err(h);
}
