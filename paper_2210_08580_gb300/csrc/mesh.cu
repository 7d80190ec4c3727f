// Non-equal-chord meshes (Sec. III-A: "L should be replaced by L~ = G^-1/2 L G^-1/2 on
// non-homogeneously discretised structures").  On such a polygon the P1 Gram matrix G and
// Laplacian L are general cyclic tridiagonal matrices,
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
//    compression), so Phi is found by shift-and-invert subspace iteration on
//    (L + sigma G)^-1 G from the arclength Fourier modes, G-orthonormalised each step by a
//    Cholesky QR, and one Rayleigh-Ritz step at the end whose small eigenproblem runs
//    through the library's one-sided Jacobi SVD.
#include <math.h>

#include <algorithm>
#include <vector>

#include "kernels.h"

// -----------------------------------------------------------------------------------------
// Bordered LDL^T of a cyclic symmetric tridiagonal matrix T with
//     T_ii = cL (1/h_{i-1} + 1/h_i) + cG (h_{i-1} + h_i)/3,
//     T_{i,i+1} = T_{i+1,i} = -cL / h_i + cG h_i / 6       (indices mod N)
// Factor layout (4 N doubles): l[i] (i = 1..N-2, subdiagonal of L), dinv[i] = 1/d_i,
// m[i] (i = 0..N-2, L's last row), sdinv[i] = d_i^-1/2.  Sequential, one thread: O(N).
// -----------------------------------------------------------------------------------------
__device__ __forceinline__ double tri_diag(const double* h, int N, int i, double cL, double cG) {
    const double hp = h[i == 0 ? N - 1 : i - 1], hi = h[i];
    return cL * (1.0 / hp + 1.0 / hi) + cG * (hp + hi) * (1.0 / 3.0);
}
__device__ __forceinline__ double tri_off(const double* h, int i, double cL, double cG) {
    return -cL / h[i] + cG * h[i] * (1.0 / 6.0);
}

__global__ void k_cyc_factor(const double* __restrict__ h, int N, double cL, double cG, double* fac, int* err) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double* l = fac;
    double* dinv = fac + N;
    double* m = fac + 2 * N;
    double* sd = fac + 3 * N;
    // border column: c_0 = T_{0,N-1}, c_{N-2} = T_{N-2,N-1} (both on the same entry when N = 2)
    const double c0 = tri_off(h, N - 1, cL, cG), cl = tri_off(h, N - 2, cL, cG);
    double d = tri_diag(h, N, 0, cL, cG);
    double z = c0;                       // z = L'^-1 c, running
    double schur = 0.0;                  // sum z_i^2 / d_i
    bool bad = !(d > 0.0);
    l[0] = 0.0;
    for (int i = 0;; ++i) {
        const double di = 1.0 / d;
        dinv[i] = di;
        sd[i] = sqrt(di);
        m[i] = z * di;
        schur += z * z * di;
        if (i == N - 2) break;
        const double b = tri_off(h, i, cL, cG);
        const double li = b * di;
        l[i + 1] = li;
        d = tri_diag(h, N, i + 1, cL, cG) - li * b;
        bad |= !(d > 0.0);
        z = ((i + 1 == N - 2) ? cl : 0.0) - li * z;
    }
    const double dl = tri_diag(h, N, N - 1, cL, cG) - schur;
    bad |= !(dl > 0.0);
    l[N - 1] = 0.0;
    m[N - 1] = 0.0;
    dinv[N - 1] = 1.0 / dl;
    sd[N - 1] = sqrt(1.0 / dl);
    if (bad) atomicOr(err, DEVERR_SINGULAR);
}

// -----------------------------------------------------------------------------------------
// Solves along index i of a strided array (element i of column c at c*sc + i*si), one thread
// per column.  MODE 0: y = scale T^-1 x (forward L, diagonal, backward L^T).  MODE 1:
// y = scale D^-1/2 L^-1 x, i.e. the rows b F^-1 with F = D^1/2 L^T (F^T F = T).  In place
// allowed (each element is read before it is written).
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
__device__ __forceinline__ cplx tsub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <> __device__ __forceinline__ cplx zero_of<cplx>() { return cmk(0, 0); }

template <typename T, int MODE>
__global__ void __launch_bounds__(64) k_cyc_solve(const T* in, T* out, int64_t N, int64_t ncols, int64_t si,
                                                  int64_t sc, const double* __restrict__ fac, double scale,
                                                  int conj_out) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const double* l = fac;
    const double* dinv = fac + N;
    const double* m = fac + 2 * N;
    const double* sd = fac + 3 * N;
    const T* x = in + col * sc;
    T* y = out + col * sc;
    // forward: u_0 = x_0, u_i = x_i - l_i u_{i-1} (i <= N-2), u_{N-1} = x_{N-1} - sum m_i u_i
    T prev = x[0];
    T s = zero_of<T>();
    s = fma_acc(s, m[0], prev);
    if (MODE == 0) y[0] = sc_mul(prev, dinv[0]);
    else y[0] = maybe_conj(sc_mul(prev, scale * sd[0]), conj_out);
    for (int64_t i = 1; i < N - 1; ++i) {
        const T u = axmy(x[i * si], l[i], prev);
        s = fma_acc(s, m[i], u);
        if (MODE == 0) y[i * si] = sc_mul(u, dinv[i]);
        else y[i * si] = maybe_conj(sc_mul(u, scale * sd[i]), conj_out);
        prev = u;
    }
    const T ul = tsub(x[(N - 1) * si], s);
    if (MODE == 1) {
        y[(N - 1) * si] = maybe_conj(sc_mul(ul, scale * sd[N - 1]), conj_out);
        return;
    }
    // backward: y_{N-1} = w_{N-1}; y_{N-2} = w_{N-2} - m_{N-2} y_{N-1};
    // y_i = w_i - l_{i+1} y_{i+1} - m_i y_{N-1}
    const T yl = sc_mul(ul, dinv[N - 1]);
    y[(N - 1) * si] = maybe_conj(sc_mul(yl, scale), conj_out);
    T next = axmy(y[(N - 2) * si], m[N - 2], yl);
    y[(N - 2) * si] = maybe_conj(sc_mul(next, scale), conj_out);
    for (int64_t i = N - 3; i >= 0; --i) {
        const T v = axmy(axmy(y[i * si], l[i + 1], next), m[i], yl);
        y[i * si] = maybe_conj(sc_mul(v, scale), conj_out);
        next = v;
    }
}

// y = T x for the cyclic tridiagonal T above, on the columns of real N x ncols (ld N)
__global__ void k_tri_mul(const double* __restrict__ x, double* __restrict__ y, int64_t N, int64_t ncols,
                          const double* __restrict__ h, double cL, double cG) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * ncols) return;
    const int64_t i = idx % N, c = idx / N;
    const int n = (int)N;
    const int ip = (i == 0) ? n - 1 : (int)i - 1, in = (i == N - 1) ? 0 : (int)i + 1;
    const double* xc = x + c * N;
    double v = tri_diag(h, n, (int)i, cL, cG) * xc[i];
    v = fma(tri_off(h, ip, cL, cG), xc[ip], v);
    v = fma(tri_off(h, (int)i, cL, cG), xc[in], v);
    y[idx] = v;
}

// s[i] = sum_{e < i} h_e (arclength at vertex i), s[N] = perimeter; one thread, fixed order
__global__ void k_arclength(const double* __restrict__ h, int N, double* s) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double a = 0.0;
    for (int i = 0; i < N; ++i) { s[i] = a; a += h[i]; }
    s[N] = a;
}

// Starting basis of the subspace iteration: arclength Fourier modes, column c of X (N x p):
// 1, cos(2 pi m s_i / P), sin(2 pi m s_i / P) for m = 1, 2, ... (cos and sin adjacent)
__global__ void k_fourier_arc(double* X, int64_t N, int64_t p, const double* __restrict__ s) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * p) return;
    const int64_t i = idx % N;
    const int c = (int)(idx / N);
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
// Real FP64 GEMM, C = alpha op(A) op(B) + beta C (column-major), 64 x 64 tiles, 16-deep K
// slices in shared memory, 4 x 4 outputs per thread.  The basis iteration's products.
// -----------------------------------------------------------------------------------------
template <int OPA, int OPB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int Nc, int K, double alpha, const double* __restrict__ A,
                                               int64_t lda, const double* __restrict__ B, int64_t ldb, double beta,
                                               double* C, int64_t ldc) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int mm, kk;
            if (OPA == OP_N) { mm = t % 64; kk = t / 64 + 4 * s; } else { kk = t % 16; mm = t / 16 + 16 * s; }
            const int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < K) v = (OPA == OP_N) ? A[gm + (int64_t)gk * lda] : A[gk + (int64_t)gm * lda];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int kk, nn;
            if (OPB == OP_N) { kk = t % 16; nn = t / 16 + 16 * s; } else { nn = t % 64; kk = t / 64 + 4 * s; }
            const int gk = k0 + kk, gn = n0 + nn;
            double v = 0.0;
            if (gk < K && gn < Nc) v = (OPB == OP_N) ? B[gk + (int64_t)gn * ldb] : B[gn + (int64_t)gk * ldb];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
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
            double* cp = C + gm + (int64_t)gn * ldc;
            *cp = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *cp);
        }
    }
}

// -----------------------------------------------------------------------------------------
// One CTA: upper Cholesky factor of a small SPD matrix, C + shift I = R^T R (R in C's upper
// triangle, in place; C column-major, ld p), and, with want_inv, Rinv = R^-1 (upper, the
// strict lower part zeroed).  A pivot that is not positive sets DEVERR_SINGULAR (and is
// replaced by 1 so the kernel finishes).  Rc, when given, receives R as complex (strict
// lower part zero), the input form of the Jacobi SVD.
// -----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_chol_inv(double* C, int p, double shift, double* Rinv, cplx* Rc, int* err) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    __shared__ double s_rjj;
    if (shift != 0.0)
        for (int j = tid; j < p; j += nt) C[j + (int64_t)j * p] += shift;
    __syncthreads();
    for (int j = 0; j < p; ++j) {
        if (tid == 0) {
            double v = C[j + (int64_t)j * p];
            if (!(v > 0.0)) { atomicOr(err, DEVERR_SINGULAR); v = 1.0; }
            v = sqrt(v);
            C[j + (int64_t)j * p] = v;
            s_rjj = v;
        }
        __syncthreads();
        const double ir = 1.0 / s_rjj;
        for (int k = j + 1 + tid; k < p; k += nt) C[j + (int64_t)k * p] *= ir;
        __syncthreads();
        // trailing update of the upper triangle: C_ik -= R_ji R_jk (j < i <= k)
        for (int k = j + 1 + warp; k < p; k += nw) {
            const double rjk = C[j + (int64_t)k * p];
            for (int i = j + 1 + lane; i <= k; i += 32) C[i + (int64_t)k * p] = fma(-C[j + (int64_t)i * p], rjk, C[i + (int64_t)k * p]);
        }
        __syncthreads();
    }
    if (Rc)
        for (int64_t idx = tid; idx < (int64_t)p * p; idx += nt) {
            const int i = (int)(idx % p), k = (int)(idx / p);
            Rc[idx] = cmk(i <= k ? C[idx] : 0.0, 0.0);
        }
    if (!Rinv) return;
    // column j of R^-1 by back substitution (one thread per column)
    for (int j = tid; j < p; j += nt) {
        double* x = Rinv + (int64_t)j * p;
        for (int i = j + 1; i < p; ++i) x[i] = 0.0;
        x[j] = 1.0 / C[j + (int64_t)j * p];
        for (int i = j - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int k = i + 1; k <= j; ++k) acc = fma(C[i + (int64_t)k * p], x[k], acc);
            x[i] = -acc / C[i + (int64_t)i * p];
        }
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
    BEM_TIMED(h, "k_cyc_factor", (k_cyc_factor<<<1, 1, 0, h->stream>>>(h->seg + 4 * h->N, (int)h->N, cL, cG, fac, h->dev_err)));
    BEM_LAUNCH(h, "k_cyc_factor");
    return BEM_OK;
}

bem_status general_gram_apply(bem_ctx* h, int mode, const cplx* in, cplx* out, int64_t N, int64_t ncols,
                              int64_t si, int64_t sc, bool conj_out) {
    if (!h->gfac) return bem_fail(h, BEM_E_INVALID, "Gram solve: no factor of the general Gram matrix");
    const unsigned blocks = (unsigned)((ncols + 63) / 64);
    if (mode == 0) {
        BEM_TIMED(h, "k_cyc_solve", (k_cyc_solve<cplx, 0><<<blocks, 64, 0, h->stream>>>(in, out, N, ncols, si, sc, h->gfac,
                                                                                      1.0, conj_out ? 1 : 0)));
    } else {
        BEM_TIMED(h, "k_cyc_solve", (k_cyc_solve<cplx, 1><<<blocks, 64, 0, h->stream>>>(in, out, N, ncols, si, sc, h->gfac,
                                                                                      1.0, conj_out ? 1 : 0)));
    }
    BEM_LAUNCH(h, "k_cyc_solve");
    return BEM_OK;
}

static bem_status dgemm(bem_ctx* h, int opa, int opb, int64_t M, int64_t Nc, int64_t K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((Nc + 63) / 64));
    if (opa == OP_T && opb == OP_N) {
        BEM_TIMED(h, "k_dgemm", (k_dgemm<OP_T, OP_N><<<grid, 256, 0, h->stream>>>((int)M, (int)Nc, (int)K, alpha, A, lda, B, ldb,
                                                                                   beta, C, ldc)));
    } else {
        BEM_TIMED(h, "k_dgemm", (k_dgemm<OP_N, OP_N><<<grid, 256, 0, h->stream>>>((int)M, (int)Nc, (int)K, alpha, A, lda, B, ldb,
                                                                                   beta, C, ldc)));
    }
    BEM_LAUNCH(h, "k_dgemm");
    return BEM_OK;
}

static bem_status tri_mul(bem_ctx* h, const double* x, double* y, int64_t ncols, double cL, double cG) {
    const int64_t tot = h->N * ncols;
    BEM_TIMED(h, "k_tri_mul", (k_tri_mul<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(x, y, h->N, ncols,
                                                                                             h->seg + 4 * h->N, cL, cG)));
    BEM_LAUNCH(h, "k_tri_mul");
    return BEM_OK;
}

// block size of the subspace iteration for n wanted pairs, and its iteration count
void general_basis_plan(int64_t N, int64_t n, double perimeter, int64_t* p_out, int* iters_out, double* sigma_out) {
    int64_t p = 2 * n + 9;
    if (p > 1023) p = 1023;
    if (p > N - 1) p = N - 1;
    if (p < n) p = n;
    // rates from the curve's Laplace-Beltrami spectrum lambda = (2 pi m / P)^2, which the
    // pencil's low eigenvalues approach (and exceed) on any mesh that resolves them
    const double w = 2.0 * BEM_PI / perimeter;
    const double mn = (double)((n - 1) / 2 + 1), mp = (double)((p + 1) / 2);
    const double lam_n = (w * mn) * (w * mn), lam_p = (w * mp) * (w * mp);
    const double sigma = std::max(0.25 * lam_n, w * w);
    const double rate = (lam_n + sigma) / (lam_p + sigma);
    int it = (rate < 1.0) ? (int)ceil(log(1e-17) / log(rate)) + 2 : 400;
    *p_out = p;
    *iters_out = std::min(std::max(it, 3), 400);
    *sigma_out = sigma;
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
    double sigma;
    general_basis_plan(N, n, h->hbar * (double)N, &p, &iters, &sigma);
    double *X = nullptr, *Y = nullptr, *Z = nullptr, *C = nullptr, *Rinv = nullptr, *Cf = nullptr, *fac = nullptr,
           *s = nullptr, *sig = nullptr;
    cplx *Rc = nullptr, *E = nullptr;
    int* perm = nullptr;
    void* jac = nullptr;
    WorkParts cv;
    cv.add((void**)&X, sizeof(double) * N * p);
    cv.add((void**)&Y, sizeof(double) * N * p);
    cv.add((void**)&Z, sizeof(double) * N * p);
    cv.add((void**)&C, sizeof(double) * p * p);
    cv.add((void**)&Rinv, sizeof(double) * p * p);
    cv.add((void**)&Cf, sizeof(double) * p * nc);
    cv.add((void**)&fac, sizeof(double) * 4 * N);
    cv.add((void**)&s, sizeof(double) * (N + 1));
    cv.add((void**)&sig, sizeof(double) * p);
    cv.add((void**)&Rc, sizeof(cplx) * p * p);
    cv.add((void**)&E, sizeof(cplx) * p * p);
    cv.add((void**)&perm, sizeof(int) * p);
    cv.add(&jac, jacobi_scratch_bytes((int)p));
    bem_status st;
    if ((st = cv.commit(h)) != BEM_OK) return st;
    // (L + sigma G) = L D L^T for the shift-and-invert steps
    if ((st = launch_cyc_factor(h, 1.0, sigma, fac)) != BEM_OK) return st;
    BEM_TIMED(h, "k_arclength", (k_arclength<<<1, 1, 0, h->stream>>>(h->seg + 4 * N, (int)N, s)));
    BEM_LAUNCH(h, "k_arclength");
    BEM_TIMED(h, "k_fourier_arc", (k_fourier_arc<<<(unsigned)((N * p + 255) / 256), 256, 0, h->stream>>>(X, N, p, s)));
    BEM_LAUNCH(h, "k_fourier_arc");
    // G-orthonormalise the columns of `in` into `out`: R^T R = in^T G in, out = in R^-1
    auto cholqr = [&](const double* in, double* out) -> bem_status {
        bem_status q;
        if ((q = tri_mul(h, in, Z, p, 0.0, 1.0)) != BEM_OK) return q;
        if ((q = dgemm(h, OP_T, OP_N, p, p, N, 1.0, in, N, Z, N, 0.0, C, p)) != BEM_OK) return q;
        BEM_TIMED(h, "k_chol_inv", (k_chol_inv<<<1, 1024, 0, h->stream>>>(C, (int)p, 0.0, Rinv, nullptr, h->dev_err)));
        BEM_LAUNCH(h, "k_chol_inv");
        return dgemm(h, OP_N, OP_N, N, p, p, 1.0, in, N, Rinv, p, 0.0, out, N);
    };
    if ((st = cholqr(X, Y)) != BEM_OK) return st;
    std::swap(X, Y);
    const unsigned sblocks = (unsigned)((p + 63) / 64);
    for (int it = 0; it < iters; ++it) {
        // Y = (L + sigma G)^-1 G X
        if ((st = tri_mul(h, X, Z, p, 0.0, 1.0)) != BEM_OK) return st;
        BEM_TIMED(h, "k_cyc_solve", (k_cyc_solve<double, 0><<<sblocks, 64, 0, h->stream>>>(Z, Y, N, p, 1, N, fac, 1.0, 0)));
        BEM_LAUNCH(h, "k_cyc_solve");
        if ((st = cholqr(Y, X)) != BEM_OK) return st;
    }
    // a second Cholesky QR restores G-orthonormality to rounding
    if ((st = cholqr(X, Y)) != BEM_OK) return st;
    std::swap(X, Y);
    // Rayleigh-Ritz: A = X^T L X; the eigenvectors of A + sigma I are the right singular
    // vectors of its Cholesky factor (Jacobi SVD, sorted by decreasing singular value)
    if ((st = tri_mul(h, X, Z, p, 1.0, 0.0)) != BEM_OK) return st;
    if ((st = dgemm(h, OP_T, OP_N, p, p, N, 1.0, X, N, Z, N, 0.0, C, p)) != BEM_OK) return st;
    BEM_TIMED(h, "k_chol_inv", (k_chol_inv<<<1, 1024, 0, h->stream>>>(C, (int)p, sigma, nullptr, Rc, h->dev_err)));
    BEM_LAUNCH(h, "k_chol_inv");
    BEM_TIMED(h, "k_iota", (k_iota<<<(unsigned)((p + 255) / 256), 256, 0, h->stream>>>(perm, (int)p)));
    BEM_LAUNCH(h, "k_iota");
    if ((st = launch_jacobi_svd(h, Rc, (int)p, perm, sig, E, jac)) != BEM_OK) return st;
    // the n lowest Ritz vectors are the last n columns; without the kernel mode the very last
    // (the constant vector, lambda = 0) is left out
    BEM_TIMED(h, "k_take_cols", (k_take_cols<<<(unsigned)((p * nc + 255) / 256), 256, 0, h->stream>>>(E, (int)p, (int)(p - n),
                                                                                                   (int)nc, Cf, h->gm)));
    BEM_LAUNCH(h, "k_take_cols");
    if ((st = dgemm(h, OP_N, OP_N, N, nc, p, 1.0, X, N, Cf, p, 0.0, h->Q, N)) != BEM_OK) return st;
    if ((st = tri_mul(h, h->Q, h->GQ, nc, 0.0, 1.0)) != BEM_OK) return st;
    return read_basis_err(h);
}
