// Dense FP64 building blocks of the filter, compression and Woodbury stages (Sec. III-IV):
//   - complex (and real x complex) GEMM on the FP64 CUDA cores,
//   - G^-1 and the Gram square-root factor applied as two first-order recursions
//     (the equal-chord Gram matrix is circulant: G = (h/6)(Z + 4 + Z^-1) =
//      (h/(6 r))(I + r Z)(I + r Z^-1), r = 2 - sqrt 3),
//   - the Fourier filter basis,
//   - Householder QR of a tall-skinny matrix and one-sided Jacobi SVD (cooperative
//     kernels with bounded grid barriers), Gauss-Jordan inversion of the Woodbury core.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "dfloat.cuh"
#include "kernels.h"

// =========================================================================================
// GEMM: C = alpha op(A) op(B) + beta C, column-major, 64x64 tiles, 16-deep K slices
// =========================================================================================
template <int OPA, int OPB, bool AREAL>
__global__ void __launch_bounds__(256) k_zgemm(int M, int Nc, int K, cplx alpha, const void* Av,
                                               int64_t lda, const cplx* B, int64_t ldb, cplx beta,
                                               cplx* C, int64_t ldc) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ cplx Bs[BK][BN];
    __shared__ typename std::conditional<AREAL, double, cplx>::type As[BK][BM];
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    cplx acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmk(0, 0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int mm, kk;
            if (OPA == OP_N) { mm = t % 64; kk = t / 64 + 4 * s; } else { kk = t % 16; mm = t / 16 + 16 * s; }
            const int gm = m0 + mm, gk = k0 + kk;
            if (AREAL) {
                const double* A = reinterpret_cast<const double*>(Av);
                double v = 0.0;
                if (gm < M && gk < K) v = (OPA == OP_N) ? A[gm + (int64_t)gk * lda] : A[gk + (int64_t)gm * lda];
                reinterpret_cast<double*>(&As[0][0])[kk * BM + mm] = v;
            } else {
                const cplx* A = reinterpret_cast<const cplx*>(Av);
                cplx v = cmk(0, 0);
                if (gm < M && gk < K) {
                    v = (OPA == OP_N) ? A[gm + (int64_t)gk * lda] : A[gk + (int64_t)gm * lda];
                    if (OPA == OP_C) v.y = -v.y;
                }
                reinterpret_cast<cplx*>(&As[0][0])[kk * BM + mm] = v;
            }
        }
        // B tile
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int kk, nn;
            if (OPB == OP_N) { kk = t % 16; nn = t / 16 + 16 * s; } else { nn = t % 64; kk = t / 64 + 4 * s; }
            const int gk = k0 + kk, gn = n0 + nn;
            cplx v = cmk(0, 0);
            if (gk < K && gn < Nc) {
                v = (OPB == OP_N) ? B[gk + (int64_t)gn * ldb] : B[gn + (int64_t)gk * ldb];
                if (OPB == OP_C) v.y = -v.y;
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            cplx b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
            if (AREAL) {
                double a[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = reinterpret_cast<const double*>(&As[0][0])[kk * BM + tx + 16 * i];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[i][j].x = fma(a[i], b[j].x, acc[i][j].x);
                        acc[i][j].y = fma(a[i], b[j].y, acc[i][j].y);
                    }
            } else {
                cplx a[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = reinterpret_cast<const cplx*>(&As[0][0])[kk * BM + tx + 16 * i];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
            }
        }
        __syncthreads();
    }
    const bool zb = (beta.x == 0.0 && beta.y == 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tx + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + ty + 16 * j;
            if (gn >= Nc) continue;
            cplx* cp = C + gm + (int64_t)gn * ldc;
            cplx v = cmul(alpha, acc[i][j]);
            if (!zb) v = cadd(v, cmul(beta, *cp));
            *cp = v;
        }
    }
}

template <int OPA, int OPB, bool AREAL>
static void zgemm_launch(cudaStream_t st, int64_t M, int64_t Nc, int64_t K, cplx alpha, const void* A,
                         int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc) {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((Nc + 63) / 64));
    k_zgemm<OPA, OPB, AREAL><<<grid, 256, 0, st>>>((int)M, (int)Nc, (int)K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// C = A B (no transposes; column-major complex FP64 in and out) with double-float
// products and sums on the FP32 pipe: 32 x 32 output tiles, K in steps of 16 staged in
// shared memory, each thread four outputs of one column.  For the small dense products of
// the mixed path (the r x r Woodbury core times r x nrhs), where FP64 issue dominates.
#define ZDF_T 32
#define ZDF_K 16
__global__ void __launch_bounds__(256) k_zgemm_df(int64_t M, int64_t Nc, int64_t K, const cplx* __restrict__ A,
                                                  int64_t lda, const cplx* __restrict__ B, int64_t ldb, cplx* C,
                                                  int64_t ldc) {
    __shared__ float4 sA[ZDF_K][ZDF_T + 1];     // [k][row]
    __shared__ float4 sB[ZDF_T][ZDF_K + 1];     // [col][k]
    const int64_t i0 = (int64_t)blockIdx.x * ZDF_T, j0 = (int64_t)blockIdx.y * ZDF_T;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // row tx, columns ty + 8 q
    cdfl acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = cdfl_zero();
    for (int64_t k0 = 0; k0 < K; k0 += ZDF_K) {
        for (int e = threadIdx.x; e < ZDF_T * ZDF_K; e += 256) {
            const int r = e % ZDF_T, kk = e / ZDF_T;
            const int64_t gi = i0 + r, gk = k0 + kk;
            const cplx a = (gi < M && gk < K) ? A[gi + gk * lda] : cmk(0, 0);
            sA[kk][r] = cdfl_pack({dfl_from_bits(a.x), dfl_from_bits(a.y)});
            const int kb = e % ZDF_K, cb = e / ZDF_K;
            const int64_t gj = j0 + cb, gk2 = k0 + kb;
            const cplx b = (gj < Nc && gk2 < K) ? B[gk2 + gj * ldb] : cmk(0, 0);
            sB[cb][kb] = cdfl_pack({dfl_from_bits(b.x), dfl_from_bits(b.y)});
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < ZDF_K; ++kk) {
            const cdfl a = cdfl_unpack(sA[kk][tx]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const cdfl b = cdfl_unpack(sB[ty + 8 * q][kk]);
                acc[q].re = dfl_fma(a.re, b.re, dfl_fma(dfl_neg(a.im), b.im, acc[q].re));
                acc[q].im = dfl_fma(a.re, b.im, dfl_fma(a.im, b.re, acc[q].im));
            }
        }
        __syncthreads();
    }
    const int64_t gi = i0 + tx;
    if (gi >= M) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t gj = j0 + ty + 8 * q;
        if (gj < Nc) C[gi + gj * ldc] = cdfl_to(acc[q]);
    }
}
bem_status zgemm_df(bem_ctx* h, int64_t M, int64_t Nc, int64_t K, const cplx* A, int64_t lda, const cplx* B,
                    int64_t ldb, cplx* C, int64_t ldc) {
    if (M <= 0 || Nc <= 0) return BEM_OK;
    if ((Nc + ZDF_T - 1) / ZDF_T > 65535) return bem_fail(h, BEM_E_UNSUPPORTED, "zgemm_df: too many columns");
    dim3 grid((unsigned)((M + ZDF_T - 1) / ZDF_T), (unsigned)((Nc + ZDF_T - 1) / ZDF_T));
    BEM_TIMED(h, h->tag, (k_zgemm_df<<<grid, 256, 0, h->stream>>>(M, Nc, K, A, lda, B, ldb, C, ldc)));
    h->tag = "kernel";
    BEM_LAUNCH(h, "k_zgemm_df");
    return BEM_OK;
}

bem_status zgemm(bem_ctx* h, int opa, int opb, int64_t M, int64_t Nc, int64_t K, cplx alpha,
                 const cplx* A, int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc) {
    if (M <= 0 || Nc <= 0) return BEM_OK;
    if (K <= 0) { K = 0; }
    cudaStream_t st = h->stream;
#define ZG(a, b) if (opa == a && opb == b) zgemm_launch<a, b, false>(st, M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc)
    BEM_TIMED(h, h->tag,
    ZG(OP_N, OP_N); else ZG(OP_N, OP_T); else ZG(OP_N, OP_C);
    else ZG(OP_T, OP_N); else ZG(OP_T, OP_T); else ZG(OP_T, OP_C);
    else ZG(OP_C, OP_N); else ZG(OP_C, OP_T); else ZG(OP_C, OP_C));
#undef ZG
    BEM_LAUNCH(h, "k_zgemm");
    return BEM_OK;
}

bem_status dzgemm_realA(bem_ctx* h, int opa, int64_t M, int64_t Nc, int64_t K, double alpha,
                        const double* A, int64_t lda, const cplx* B, int64_t ldb, double beta,
                        cplx* C, int64_t ldc) {
    if (M <= 0 || Nc <= 0) return BEM_OK;
    BEM_TIMED(h, h->tag,
    if (opa == OP_N)
        zgemm_launch<OP_N, OP_N, true>(h->stream, M, Nc, K, cmk(alpha, 0), A, lda, B, ldb, cmk(beta, 0), C, ldc);
    else
        zgemm_launch<OP_T, OP_N, true>(h->stream, M, Nc, K, cmk(alpha, 0), A, lda, B, ldb, cmk(beta, 0), C, ldc));
    BEM_LAUNCH(h, "k_dzgemm");
    return BEM_OK;
}

// =========================================================================================
// Gram recursions.  r = 2 - sqrt(3), |r|^33 < 1e-18: a chunk's first output is seeded with
// the truncated lookback sum y_i0 = sum_{j<33} (-r)^j x_{i0 -/+ j} (periodic indices).
// =========================================================================================
#define IIR_CHUNK 32
#define IIR_LOOK 33

__global__ void k_iir(const cplx* __restrict__ in, cplx* __restrict__ out, int64_t N, int64_t ncols,
                      int64_t si, int64_t sc, double r, int dir, double scale, int conj_out) {
    const int64_t nchunk = (N + IIR_CHUNK - 1) / IIR_CHUNK;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t col, ch;
    if (sc == 1) { col = tid % ncols; ch = tid / ncols; } else { ch = tid % nchunk; col = tid / nchunk; }
    if (col >= ncols || ch >= nchunk) return;
    const cplx* x = in + col * sc;
    cplx* y = out + col * sc;
    const int64_t a = ch * IIR_CHUNK, b = min(N, a + IIR_CHUNK);
    if (dir > 0) {
        cplx acc = cmk(0, 0);
        double c = 1.0;
        for (int j = 0; j < IIR_LOOK; ++j) {
            int64_t ii = a - j;                  // >= -IIR_LOOK: wrapped by adding N
            while (ii < 0) ii += N;
            const cplx v = x[ii * si];
            acc.x += c * v.x; acc.y += c * v.y;
            c *= -r;
        }
        cplx prev = acc;
        y[a * si] = cmk(scale * prev.x, conj_out ? -scale * prev.y : scale * prev.y);
        for (int64_t i = a + 1; i < b; ++i) {
            const cplx v = x[i * si];
            prev = cmk(v.x - r * prev.x, v.y - r * prev.y);
            y[i * si] = cmk(scale * prev.x, conj_out ? -scale * prev.y : scale * prev.y);
        }
    } else {
        const int64_t last = b - 1;
        cplx acc = cmk(0, 0);
        double c = 1.0;
        for (int j = 0; j < IIR_LOOK; ++j) {
            int64_t ii = last + j;               // < N + IIR_LOOK: wrapped by subtracting N
            while (ii >= N) ii -= N;
            const cplx v = x[ii * si];
            acc.x += c * v.x; acc.y += c * v.y;
            c *= -r;
        }
        cplx prev = acc;
        y[last * si] = cmk(scale * prev.x, conj_out ? -scale * prev.y : scale * prev.y);
        for (int64_t i = last - 1; i >= a; --i) {
            const cplx v = x[i * si];
            prev = cmk(v.x - r * prev.x, v.y - r * prev.y);
            y[i * si] = cmk(scale * prev.x, conj_out ? -scale * prev.y : scale * prev.y);
        }
    }
}

bem_status apply_gram_inverse(bem_ctx* h, int mode, const cplx* in, cplx* out, cplx* tmp, int64_t N,
                              int64_t ncols, int64_t si, int64_t sc, double hbar, bool conj_out) {
    // on a general mesh tmp (when given) holds at least N ncols elements: the chunked solves' scratch
    if (h->general) return general_gram_apply(h, mode, in, out, tmp, tmp ? (size_t)(N * ncols) : 0, N, ncols, si, sc, conj_out);
    const double r = 2.0 - sqrt(3.0);
    const int64_t nchunk = (N + IIR_CHUNK - 1) / IIR_CHUNK;
    const int64_t threads = nchunk * ncols;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (mode == 0) {
        // G^-1 = (6 r / h) (I + r Z)^-1 (I + r Z^-1)^-1
        BEM_TIMED(h, "k_iir", (k_iir<<<blocks, 256, 0, h->stream>>>(in, tmp, N, ncols, si, sc, r, +1, 1.0, 0)));
        BEM_TIMED(h, "k_iir", (k_iir<<<blocks, 256, 0, h->stream>>>(tmp, out, N, ncols, si, sc, r, -1,
                                                                    6.0 * r / hbar, conj_out ? 1 : 0)));
    } else {
        // F^-T with G = F^T F, F = sqrt(h/(6r)) (I + r Z^-1): one causal pass
        BEM_TIMED(h, "k_iir", (k_iir<<<blocks, 256, 0, h->stream>>>(in, out, N, ncols, si, sc, r, +1,
                                                                    sqrt(6.0 * r / hbar), conj_out ? 1 : 0)));
    }
    BEM_LAUNCH(h, "k_iir");
    return BEM_OK;
}

// =========================================================================================
// Fourier filter basis: column c of Q (N x ncols, column-major) with m = mode index:
//   constant 1/sqrt(N);  cos: sqrt(2/N) cos(2 pi m i/N);  sin: sqrt(2/N) sin(2 pi m i/N)
// (argument reduced exactly as (m i mod N)).  gm[c] = h (2 + cos(2 pi m/N))/3.
// =========================================================================================
__device__ __forceinline__ void fourier_col(int c, int include_kernel, int& m, int& is_sin) {
    if (include_kernel) {
        if (c == 0) { m = 0; is_sin = 0; return; }
        m = (c + 1) / 2; is_sin = (c % 2 == 0);
    } else {
        m = c / 2 + 1; is_sin = (c % 2 == 1);
    }
}

__global__ void k_fourier(double* Q, int64_t N, int64_t ncols, int include_kernel, double* gm, double hbar) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * ncols) return;
    const int64_t i = idx % N;
    const int c = (int)(idx / N);
    int m, is_sin;
    fourier_col(c, include_kernel, m, is_sin);
    double v;
    if (m == 0) {
        v = 1.0 / sqrt((double)N);
    } else {
        const int64_t red = ((int64_t)m * i) % N;
        double s, co;
        sincospi(2.0 * (double)red / (double)N, &s, &co);
        v = sqrt(2.0 / (double)N) * (is_sin ? s : co);
    }
    Q[i + c * N] = v;
    if (i == 0) {
        double s, co;
        sincospi(2.0 * (double)m / (double)N, &s, &co);
        gm[c] = hbar * (2.0 + co) / 3.0;
    }
}

bem_status launch_fourier_basis(bem_ctx* h, double* Q, int64_t N, int64_t ncols, int include_kernel,
                                double* gm, double hbar) {
    const int64_t tot = N * ncols;
    BEM_TIMED(h, "k_fourier", (k_fourier<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(Q, N, ncols, include_kernel, gm, hbar)));
    BEM_LAUNCH(h, "k_fourier");
    return BEM_OK;
}

// B[c, i] <- B[c, i] / g_c - Q[i, c] / 4     (B: ncols x N, ld = ncols)
__global__ void k_finish_B(cplx* B, const double* gm, const double* Q, int64_t ncols, int64_t N) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncols * N) return;
    const int64_t c = idx % ncols, i = idx / ncols;
    const double ig = 1.0 / gm[c];
    cplx v = B[idx];
    B[idx] = cmk(v.x * ig - 0.25 * Q[i + c * N], v.y * ig);
}

bem_status launch_finish_B(bem_ctx* h, cplx* B, const double* gm, const double* Q, int64_t ncols, int64_t N) {
    const int64_t tot = ncols * N;
    BEM_TIMED(h, "k_finish_B", (k_finish_B<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(B, gm, Q, ncols, N)));
    BEM_LAUNCH(h, "k_finish_B");
    return BEM_OK;
}

// out[row, col] = in[row, col] * s[row]^(pw/2)   (pw = +1: sqrt, -1: 1/sqrt, 2: s, -2: 1/s)
__device__ __forceinline__ double powsel(double s, int pw) {
    switch (pw) {
        case 1: return sqrt(s);
        case -1: return 1.0 / sqrt(s);
        case 2: return s;
        default: return 1.0 / s;
    }
}
__global__ void k_row_scale(const cplx* in, cplx* out, const double* s, int pw, int64_t rows, int64_t cols, int64_t ld) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t rr = idx % rows, cc = idx / rows;
    const double f = powsel(s[rr], pw);
    const cplx v = in[rr + cc * ld];
    out[rr + cc * ld] = cmk(v.x * f, v.y * f);
}
bem_status launch_row_scale(bem_ctx* h, const cplx* in, cplx* out, const double* s, int pw, int64_t rows,
                            int64_t cols, int64_t ld) {
    const int64_t tot = rows * cols;
    BEM_TIMED(h, "k_row_scale", (k_row_scale<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(in, out, s, pw, rows, cols, ld)));
    BEM_LAUNCH(h, "k_row_scale");
    return BEM_OK;
}
// real matrix (rows x cols, ld = rows): out[:, c] = in[:, c] * s[c]^(pw/2)
__global__ void k_scale_real_cols(const double* in, double* out, const double* s, int pw, int64_t rows, int64_t cols) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    out[idx] = in[idx] * powsel(s[idx / rows], pw);
}
bem_status launch_scale_real_cols(bem_ctx* h, const double* in, double* out, const double* s, int pw,
                                  int64_t rows, int64_t cols) {
    const int64_t tot = rows * cols;
    BEM_TIMED(h, "k_scale_real_cols", (k_scale_real_cols<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(in, out, s, pw, rows, cols)));
    BEM_LAUNCH(h, "k_scale_real_cols");
    return BEM_OK;
}

// =========================================================================================
// Householder QR of X (N x n, stored row-major: X[i*n + c]), R (n x n, column-major).
// Cooperative: CTA b owns rows [b*rb, (b+1)*rb).  Per column j: (1) partial |x|^2, barrier,
// (2) reflector from the global norm, (3) partial w_c = v^H X[:, c], barrier, (4) update.
// =========================================================================================
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < nw; ++q) s += red[q];
    return s;
}

// Householder QR with column pivoting of X (N x n, row-major, N >= n): X P = Q R.
// Rows are split evenly over the CTAs; per column two grid barriers.  Pivoting is by the
// largest trailing column norm, from per-CTA partial norms accumulated while the previous
// reflector is applied (so no extra pass over X).  For the comparison the partials are
// summed by integer atomics in 62-bit fixed point (scaled by the largest initial column
// norm; integer addition keeps the choice independent of arrival order); the reflector
// uses the FP64 sum of the chosen column's partials.  Columns are never moved:
// cmap[c] is the storage column of logical column c, identical in every CTA.  On exit
// perm[c] = cmap[c] (X P has column c = column perm[c] of X) and R (n x n, column-major)
// holds the upper triangle.  The pivoting grades R so that one-sided Jacobi on R^H needs
// few sweeps (Drmac and Veselic's preconditioned Jacobi SVD).
__global__ void __launch_bounds__(256) k_house_qr(cplx* X, int64_t N, int n, cplx* R, int* perm, double* partC,
                                                  unsigned long long* cnq, cplx* partW, unsigned* bar, int* err) {
    __shared__ double red[32];
    __shared__ cplx wred[8][33];
    __shared__ double nred[8][33];
    __shared__ cplx wsm[1024];
    __shared__ int cmap[1024];
    __shared__ double qscale_s;
    __shared__ unsigned long long pbest[8];
    __shared__ int pidx[8];
    const unsigned G = gridDim.x;
    const int64_t rb = (N + G - 1) / G;
    const int64_t r0 = (int64_t)blockIdx.x * rb, r1 = min(N, r0 + rb);
    const int tid = threadIdx.x, cg = tid & 31, rg = tid >> 5, lane = tid & 31;
    for (int c = tid; c < n; c += blockDim.x) cmap[c] = c;
    // partial column norms over my rows
    for (int cb = 0; cb < n; cb += 32) {
        const int c = cb + cg;
        double acc = 0.0;
        if (c < n)
            for (int64_t i = r0 + rg; i < r1; i += 8) acc += cabs2(X[i * n + c]);
        nred[rg][cg] = acc;
        __syncthreads();
        if (rg == 0 && c < n) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += nred[q][cg];
            partC[(int64_t)blockIdx.x * n + c] = t;
        }
        __syncthreads();
    }
    if (!grid_barrier(bar, G, err)) return;
    // fixed-point scale from the largest column norm (every CTA alike), then the first
    // pivot sums (cnq[0] and cnq[1] were zeroed before the launch)
    {
        double mx = 0.0;
        for (int c = tid; c < n; c += blockDim.x) {
            double t = 0.0;
            for (unsigned q = 0; q < G; ++q) t += partC[(int64_t)q * n + c];
            mx = fmax(mx, t);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red[rg] = mx;
        __syncthreads();
        if (tid == 0) {
            double m2 = 0.0;
            for (int q = 0; q < 8; ++q) m2 = fmax(m2, red[q]);
            qscale_s = (m2 > 0.0) ? 4.0e18 / m2 : 0.0;      // sums stay below 2^62
        }
        __syncthreads();
        for (int c = tid; c < n; c += blockDim.x)
            atomicAdd(cnq + c, __double2ull_rz(partC[(int64_t)blockIdx.x * n + c] * qscale_s));
    }
    const double qscale = qscale_s;
    for (int j = 0; j < n; ++j) {
        if (!grid_barrier(bar, G, err)) return;
        // (1) pivot: the largest trailing column norm (ties to the lower index)
        const unsigned long long* cq = cnq + (size_t)(j & 1) * n;
        unsigned long long best = 0ull;
        int bi = n;
        for (int c = j + tid; c < n; c += blockDim.x) {
            const unsigned long long v = __ldcg(cq + cmap[c]);
            if (bi == n || v > best) { best = v; bi = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi < n && (bi == n || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
        }
        if (lane == 0) { pbest[rg] = best; pidx[rg] = bi; }
        __syncthreads();
        if (tid == 0) {
            unsigned long long b2 = pbest[0];
            int i2 = pidx[0];
            for (int q = 1; q < 8; ++q)
                if (pidx[q] < n && (i2 == n || pbest[q] > b2 || (pbest[q] == b2 && pidx[q] < i2))) {
                    b2 = pbest[q]; i2 = pidx[q];
                }
            if (i2 > j && i2 < n) { const int t = cmap[j]; cmap[j] = cmap[i2]; cmap[i2] = t; }
        }
        // the other buffer collects the norms after this step's update
        if (blockIdx.x == 0)
            for (int c = tid; c < n; c += blockDim.x) cnq[(size_t)((j + 1) & 1) * n + c] = 0ull;
        __syncthreads();
        const int pj = cmap[j];
        double nrm2 = 0.0;
        for (unsigned q = tid; q < G; q += blockDim.x) nrm2 += partC[(int64_t)q * n + pj];
        nrm2 = block_sum(nrm2, red);
        // (2) reflector
        const cplx xjj = X[(int64_t)j * n + pj];
        double tau = 0.0;
        cplx alpha = cmk(0, 0), vj = cmk(0, 0);
        if (nrm2 > 0.0) {
            const double a = sqrt(nrm2), ax = sqrt(cabs2(xjj));
            const cplx ph = (ax > 0.0) ? cmk(xjj.x / ax, xjj.y / ax) : cmk(1, 0);
            alpha = cmk(-ph.x * a, -ph.y * a);
            vj = csub(xjj, alpha);
            const double vn2 = nrm2 - ax * ax + cabs2(vj);
            tau = (vn2 > 0.0) ? 2.0 / vn2 : 0.0;
        }
        if (tid == 0 && j >= r0 && j < r1) R[j + (int64_t)j * n] = (nrm2 > 0.0) ? alpha : cmk(0, 0);
        // (3) partial dots w_c = sum_i conj(v_i) X[i, c], c > j
        for (int cb = j + 1; cb < n; cb += 32) {
            const int c = cb + cg;
            cplx acc = cmk(0, 0);
            if (c < n && tau != 0.0) {
                const int pc = cmap[c];
                for (int64_t i = max(r0, (int64_t)j) + rg; i < r1; i += 8) {
                    const cplx vi = (i == j) ? vj : X[i * n + pj];
                    cfma_conj(acc, vi, X[i * n + pc]);
                }
            }
            wred[rg][cg] = acc;
            __syncthreads();
            if (rg == 0) {
                cplx t = wred[0][cg];
                for (int q = 1; q < 8; ++q) t = cadd(t, wred[q][cg]);
                if (c < n) partW[(int64_t)blockIdx.x * n + c] = t;
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, G, err)) return;
        // (4) reduce w over CTAs; update my rows and accumulate their trailing norms
        for (int c = j + 1 + tid; c < n; c += blockDim.x) {
            cplx t = cmk(0, 0);
            for (unsigned q = 0; q < G; ++q) t = cadd(t, partW[(int64_t)q * n + c]);
            wsm[c] = cscale(t, tau);
        }
        __syncthreads();
        for (int cb = j + 1; cb < n; cb += 32) {
            const int c = cb + cg;
            double acc = 0.0;
            if (c < n) {
                const int pc = cmap[c];
                const cplx wc = wsm[c];
                for (int64_t i = max(r0, (int64_t)j) + rg; i < r1; i += 8) {
                    cplx x = X[i * n + pc];
                    if (tau != 0.0) {
                        const cplx vi = (i == j) ? vj : X[i * n + pj];
                        x = csub(x, cmul(vi, wc));
                        X[i * n + pc] = x;
                    }
                    if (i > j) acc += cabs2(x);
                }
            }
            nred[rg][cg] = acc;
            __syncthreads();
            if (rg == 0 && c < n) {
                double t = 0.0;
                for (int q = 0; q < 8; ++q) t += nred[q][cg];
                partC[(int64_t)blockIdx.x * n + cmap[c]] = t;
                atomicAdd(cnq + (size_t)((j + 1) & 1) * n + cmap[c], __double2ull_rz(t * qscale));
            }
            __syncthreads();
        }
    }
    // R's rows owned here (the diagonal was written at each step)
    for (int64_t j = max(r0, (int64_t)0); j < min(r1, (int64_t)n); ++j)
        for (int c = tid; c < n; c += blockDim.x)
            if (c != j) R[j + (int64_t)c * n] = (c < j) ? cmk(0, 0) : X[j * n + cmap[c]];
    if (blockIdx.x == 0)
        for (int c = tid; c < n; c += blockDim.x) perm[c] = cmap[c];
}

static bem_status coop_launch(bem_ctx* h, const void* fn, int blocks_wanted, int threads, void** args, const char* what,
                              size_t smem = 0) {
    int dev = h->device, nsm = 0, per = 0;
    BEM_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // dynamic shared memory beyond the default 48 KB (less the static part) needs the opt-in
    if (smem > 0) BEM_CUDA(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BEM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem));
    if (per < 1) return bem_fail(h, BEM_E_CUDA, std::string(what) + ": kernel cannot be resident");
    int G = blocks_wanted;
    if (G > nsm * per) G = nsm * per;
    if (G < 1) G = 1;
    BEM_CUDA(h, cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), h->stream));
    BEM_CUDA(h, cudaLaunchCooperativeKernel(fn, dim3(G), dim3(threads), args, smem, h->stream));
    BEM_LAUNCH(h, what);
    return BEM_OK;
}

// The same pivoted QR for the mixed path with X held in double-float (float4 per complex
// entry: re.hi, re.lo, im.hi, im.lo).  Dots, updates and norms run on the FP32 pipe;
// cross-CTA partial sums are exchanged in FP64, and the reflector (a handful of FP64
// operations) is formed by one thread and shared.  Backward error about 1e-13 relative,
// far below the compression tolerances the path uses.
__device__ __forceinline__ cdfl cdfl_ld(const float4* p) { return cdfl_unpack(*p); }
__device__ __forceinline__ void cdfl_conj_fma(cdfl& acc, const cdfl& v, const cdfl& x) {   // acc += conj(v) x
    acc.re = dfl_fma(v.re, x.re, acc.re);
    acc.re = dfl_fma(v.im, x.im, acc.re);
    acc.im = dfl_fma(v.re, x.im, acc.im);
    acc.im = dfl_fma(dfl_neg(v.im), x.re, acc.im);
}

__global__ void k_to_dfl(float4* X, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double2 v = reinterpret_cast<const double2*>(X)[i];
    X[i] = cdfl_pack({dfl_from(v.x), dfl_from(v.y)});
}

// ---- exact fixed-point sums for the cross-CTA reductions of the double-float QR ----
// A float f = m 2^(e - 150) is added to an integer window whose least significant bit is
// 2^eb, held in three signed 64-bit limbs: limb l carries bits [l QX_W, (l + 1) QX_W) of
// the window (the top limb also the carries).  Each CTA adds its partials with integer
// atomics, so the total is exact and the same in any order of arrival; bits below 2^eb are
// dropped (the window spans 120 bits under the largest possible sum).
#define QX_W 40
__device__ __forceinline__ void qx_add(float f, int eb, long long& L0, long long& L1, long long& L2) {
    const unsigned b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 255u);
    if (e == 0) return;
    unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
    int sh = e - 150 - eb;                       // window position of m's lowest bit
    if (sh < 0) {
        if (sh <= -24) return;
        m >>= -sh;
        sh = 0;
    }
    const bool neg = (b >> 31) != 0;
    if (sh >= 2 * QX_W) {                        // top limb only (the window bounds sh)
        const long long v = (long long)(m << min(sh - 2 * QX_W, 38));
        L2 += neg ? -v : v;
        return;
    }
    const bool up = sh >= QX_W;
    const unsigned long long v = m << (up ? sh - QX_W : sh);     // shift < 40, m < 2^24
    long long lo = (long long)(v & ((1ull << QX_W) - 1)), hi = (long long)(v >> QX_W);
    if (neg) { lo = -lo; hi = -hi; }
    if (up) { L1 += lo; L2 += hi; } else { L0 += lo; L1 += hi; }
}
__device__ __forceinline__ float pow2f(int e) {   // 2^e, 0 below the normal range
    return (e < -126) ? 0.f : __uint_as_float((unsigned)(min(e, 127) + 127) << 23);
}
// limbs -> double-float: each limb (|L| < 2^48: at most 2^11 partials of 40-bit digits, or
// the small top limb) is an exact double-float a 2^24 + b; the three are summed in
// double-float (relative error about 2^-47 of the total)
__device__ __forceinline__ dfl qx_limb(long long L, int e) {
    const long long a = L >> 24;                 // arithmetic: L = a 2^24 + b, 0 <= b < 2^24
    const float fb = (float)(int)(L - (a << 24));
    const float fa = (float)(int)a;
    return dfl_add(dfl{fa * pow2f(e + 24), 0.f}, dfl{fb * pow2f(e), 0.f});
}
__device__ __forceinline__ dfl qx_to_dfl(const unsigned long long* L, int eb) {
    const dfl t2 = qx_limb((long long)L[2], eb + 2 * QX_W);
    const dfl t1 = qx_limb((long long)L[1], eb + QX_W);
    const dfl t0 = qx_limb((long long)L[0], eb);
    return dfl_add(t2, dfl_add(t1, t0));
}

// Pivoted Householder QR of X (N x n) in double-float with ONE grid barrier per column.
// Rows are split over the CTAs; every CTA keeps the column permutation (cmap: position ->
// column of X).  At the barrier of step j the exact sums over rows i >= j of
//   d_c = conj(x_{i,p}) x_{i,c}  (p = cmap[j], the pivot)   and   n_c = |x_{i,c}|^2
// are complete for every trailing column.  Each CTA then forms the reflector of the pivot
// (alpha = -e^{i arg x_jp} sqrt(n_p), v = x_p - alpha e_j, tau = 1/(|alpha| (|alpha| +
// |x_jp|))), w_c = tau (d_c - conj(alpha) x_jc), row j of R (R_jc = x_jc - v_j w_c), the
// downdated norms n_c - |R_jc|^2 and from them the next pivot; then it updates its rows
// (x_c -= v w_c) and, in the same pass, accumulates the sums of step j + 1 against the
// updated next pivot column.  n <= 32 QR_KC.
#define QR_KC 7
#define QR_KS ((QR_KC + 1) / 2)      // slots per thread (two column groups)
#define QR_NP (32 * QR_KC)
#define QR_NT 512
__global__ void __launch_bounds__(QR_NT, 1) k_house_qr_df(float4* X, int64_t N, int n, cplx* R, int* perm,
                                                       unsigned long long* lim, int* emax, float4* Pc, unsigned* bar,
                                                       int* err) {
    extern __shared__ float4 qsm[];
    float4* wbD = qsm;                                    // [8][QR_NP] per-warp dot partials
    float* wbN = reinterpret_cast<float*>(wbD + 8 * QR_NP);     // [8][QR_NP] norm partials (FP32)
    float4* sRow = reinterpret_cast<float4*>(wbN + 8 * QR_NP);  // [QR_NP] row j (by position)
    float4* sW = sRow + QR_NP;                            // [QR_NP] w by position
    float4* sD = sW + QR_NP;                              // [QR_NP] d by position
    float2* sN = reinterpret_cast<float2*>(sD + QR_NP);  // [QR_NP] n by position
    __shared__ int cmap[QR_NP];
    __shared__ float4 s_ref[2];                           // alpha, v_j
    __shared__ float2 s_tau;
    __shared__ float2 s_best[QR_NT / 32];
    __shared__ int s_bidx[QR_NT / 32];
    __shared__ int s_eb;
    const unsigned G = gridDim.x;
    const int64_t rb = (N + G - 1) / G;
    const int64_t r0 = (int64_t)blockIdx.x * rb, r1 = min(N, r0 + rb);
    // warp w: row group w & 7, column group w >> 3 (slots k = 2 kk + column group)
    const int tid = threadIdx.x, warp = tid >> 5, rg = warp & 7, cgp = warp >> 3, lane = tid & 31;
    const size_t LS = (size_t)n * 9;                      // limbs per buffer: 9 per column
    for (int c = tid; c < n; c += blockDim.x) cmap[c] = c;
    __syncthreads();

    // per-warp partials -> per-position sums over the CTA (df), into wbD[0] / wbN[0]
    auto reduce_warps = [&](int cnt) {
        __syncthreads();
        for (int l = tid; l < cnt; l += blockDim.x) {
            cdfl d = cdfl_unpack(wbD[l]);
            float nn = wbN[l];
            for (int q = 1; q < 8; ++q) {
                d = cdfl_add(d, cdfl_unpack(wbD[q * QR_NP + l]));
                nn += wbN[q * QR_NP + l];
            }
            wbD[l] = cdfl_pack(d);
            wbN[l] = nn;
        }
        __syncthreads();
    };
    // adds the CTA's sums for positions c0 + l (l < cnt) to buffer buf (exact, integer atomics)
    auto publish = [&](int c0, int cnt, int buf, int eb) {
        for (int l = tid; l < cnt; l += blockDim.x) {
            const float4 d = wbD[l];
            long long L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            qx_add(d.x, eb, L[0], L[1], L[2]); qx_add(d.y, eb, L[0], L[1], L[2]);
            qx_add(d.z, eb, L[3], L[4], L[5]); qx_add(d.w, eb, L[3], L[4], L[5]);
            qx_add(wbN[l], eb, L[6], L[7], L[8]);
            unsigned long long* dst = lim + (size_t)buf * LS + (size_t)cmap[c0 + l] * 9;
#pragma unroll
            for (int u = 0; u < 9; ++u)
                if (L[u]) atomicAdd(dst + u, (unsigned long long)L[u]);
        }
    };
    // one pass over this CTA's rows i >= jp1: optionally x_c -= v_i w_c for the positions
    // c >= jp1 (v_i: the pivot column as updated by the previous pass, kept in Pc), then
    // partial sums of conj(x_{i,p'}) x_{i,c} (double-float; p' = cmap[jp1], the next pivot)
    // and |x_{i,c}|^2 (FP32: the norms only choose pivots) with the updated values; leaves
    // the CTA's sums in wbD[0], wbN[0].  The next pivot column's new values go to Pc, not to
    // X, so that column of X is read-only during the pass: column group 0 has it in slot 0
    // (lane 0) and shares it by a shuffle, column group 1 recomputes it from X.
    auto pass = [&](int jp1, bool upd) {
        int pcs[QR_KS];
#pragma unroll
        for (int kk = 0; kk < QR_KS; ++kk) {
            const int k = 2 * kk + cgp, c = jp1 + lane + 32 * k;
            pcs[kk] = (k < QR_KC && c < n) ? cmap[c] : -1;
        }
        const int pn = (jp1 < n) ? cmap[jp1] : -1;
        const float4* pin = Pc + (size_t)((jp1 & 1) ^ 1) * N;
        float4* pout = Pc + (size_t)(jp1 & 1) * N;
        const cdfl wn = (upd && pn >= 0) ? cdfl_unpack(sW[jp1]) : cdfl_zero();
        cdfl accD[QR_KS];
        float accN[QR_KS];
#pragma unroll
        for (int kk = 0; kk < QR_KS; ++kk) { accD[kk] = cdfl_zero(); accN[kk] = 0.f; }
        auto upd1 = [&](cdfl x, const cdfl& vi, const cdfl& wk) {
            x.re = dfl_fma(dfl_neg(vi.re), wk.re, dfl_fma(vi.im, wk.im, x.re));
            x.im = dfl_fma(dfl_neg(vi.re), wk.im, dfl_fma(dfl_neg(vi.im), wk.re, x.im));
            return x;
        };
        // one row per iteration; the next row's loads are issued before this row's arithmetic
        auto load = [&](int64_t i, cdfl& vi, cdfl* x, cdfl& xo) {
            const bool ok = i < r1;
            vi = (upd && ok) ? cdfl_unpack(pin[i]) : cdfl_zero();
#pragma unroll
            for (int kk = 0; kk < QR_KS; ++kk) x[kk] = (ok && pcs[kk] >= 0) ? cdfl_ld(X + i * n + pcs[kk]) : cdfl_zero();
            xo = (ok && cgp == 1 && pn >= 0) ? cdfl_ld(X + i * n + pn) : cdfl_zero();
        };
        int64_t i = max(r0, (int64_t)jp1) + rg;
        cdfl vi, x[QR_KS], xo;
        load(i, vi, x, xo);
        for (; i < r1; i += 8) {
            cdfl vn, xn[QR_KS], xon;
            load(i + 8, vn, xn, xon);
            if (upd) {
#pragma unroll
                for (int kk = 0; kk < QR_KS; ++kk) {
                    if (pcs[kk] < 0) continue;
                    x[kk] = upd1(x[kk], vi, cdfl_unpack(sW[jp1 + lane + 32 * (2 * kk + cgp)]));
                    if (pcs[kk] != pn) X[i * n + pcs[kk]] = cdfl_pack(x[kk]);
                }
                if (cgp == 1 && pn >= 0) xo = upd1(xo, vi, wn);
            }
            cdfl p;
            if (cgp == 0) {
                p = {{__shfl_sync(0xffffffffu, x[0].re.hi, 0), __shfl_sync(0xffffffffu, x[0].re.lo, 0)},
                     {__shfl_sync(0xffffffffu, x[0].im.hi, 0), __shfl_sync(0xffffffffu, x[0].im.lo, 0)}};
                if (lane == 0 && pn >= 0) pout[i] = cdfl_pack(p);
            } else {
                p = xo;
            }
#pragma unroll
            for (int kk = 0; kk < QR_KS; ++kk) {
                if (pcs[kk] < 0) continue;
                cdfl_conj_fma(accD[kk], p, x[kk]);
                accN[kk] = fmaf(x[kk].re.hi, x[kk].re.hi, fmaf(x[kk].im.hi, x[kk].im.hi, accN[kk]));
            }
            vi = vn;
            xo = xon;
#pragma unroll
            for (int kk = 0; kk < QR_KS; ++kk) x[kk] = xn[kk];
        }
#pragma unroll
        for (int kk = 0; kk < QR_KS; ++kk) {
            const int k = 2 * kk + cgp;
            if (k >= QR_KC) continue;
            wbD[rg * QR_NP + lane + 32 * k] = cdfl_pack(accD[kk]);
            wbN[rg * QR_NP + lane + 32 * k] = accN[kk];
        }
        reduce_warps(n - jp1);
    };
    // argmax over positions [c0, n) of the df values in sN (ties: lowest position)
    auto pick = [&](int c0) -> int {
        float2 best = make_float2(-1.f, 0.f);
        int bi = n;
        for (int c = c0 + tid; c < n; c += blockDim.x) {
            const float2 v = sN[c];
            if (bi == n || v.x > best.x || (v.x == best.x && v.y > best.y)) { best = v; bi = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ox = __shfl_xor_sync(0xffffffffu, best.x, o), oy = __shfl_xor_sync(0xffffffffu, best.y, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            const bool better = oi < n && (bi == n || ox > best.x || (ox == best.x && (oy > best.y || (oy == best.y && oi < bi))));
            if (better) { best = make_float2(ox, oy); bi = oi; }
        }
        if (lane == 0) { s_best[warp] = best; s_bidx[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            float2 b2 = s_best[0];
            int i2 = s_bidx[0];
            for (int q = 1; q < QR_NT / 32; ++q) {
                const float2 v = s_best[q];
                const int qi = s_bidx[q];
                if (qi < n && (i2 == n || v.x > b2.x || (v.x == b2.x && (v.y > b2.y || (v.y == b2.y && qi < i2))))) {
                    b2 = v; i2 = qi;
                }
            }
            s_bidx[0] = i2;
        }
        __syncthreads();
        return s_bidx[0];
    };

    // ---- start: window exponent from the largest partial column norm, then the norms,
    // the first pivot and the sums of step 0
    {
        int pcs[QR_KS];
        float acc[QR_KS];
#pragma unroll
        for (int kk = 0; kk < QR_KS; ++kk) {
            const int k = 2 * kk + cgp, c = lane + 32 * k;
            pcs[kk] = (k < QR_KC && c < n) ? c : -1;
            acc[kk] = 0.f;
        }
        for (int64_t i = r0 + rg; i < r1; i += 8) {
#pragma unroll
            for (int kk = 0; kk < QR_KS; ++kk)
                if (pcs[kk] >= 0) {
                    const float4 x = X[i * n + pcs[kk]];
                    acc[kk] = fmaf(x.x, x.x, fmaf(x.z, x.z, acc[kk]));
                }
        }
#pragma unroll
        for (int kk = 0; kk < QR_KS; ++kk) {
            const int k = 2 * kk + cgp;
            if (k >= QR_KC) continue;
            wbD[rg * QR_NP + lane + 32 * k] = make_float4(0.f, 0.f, 0.f, 0.f);
            wbN[rg * QR_NP + lane + 32 * k] = acc[kk];
        }
        reduce_warps(n);
        int mx = 0;
        for (int c = tid; c < n; c += blockDim.x) mx = max(mx, (int)((__float_as_uint(wbN[c]) >> 23) & 255u));
        mx = __reduce_max_sync(0xffffffffu, (unsigned)mx);
        if (lane == 0 && mx) atomicMax(emax, mx);
    }
    if (!grid_barrier(bar, G, err)) return;
    if (tid == 0) {
        // every partial is below 2^(F + 1), F = the largest biased field - 127; sums of up
        // to 2^11 of them stay below 2^(F + 12), the top of the window
        const int F = __ldcg(emax) - 127;
        s_eb = F + 12 - 3 * QX_W;
    }
    __syncthreads();
    const int eb = s_eb;
    publish(0, n, 2, eb);                                 // norms -> buffer 2 (dots there are 0)
    if (!grid_barrier(bar, G, err)) return;
    for (int c = tid; c < n; c += blockDim.x) {
        unsigned long long Lv[3];
        const unsigned long long* src = lim + 2 * LS + (size_t)c * 9 + 6;
        for (int u = 0; u < 3; ++u) Lv[u] = __ldcg(src + u);
        const dfl v = qx_to_dfl(Lv, eb);
        sN[c] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    {
        const int q = pick(0);
        if (tid == 0 && q < n && q != 0) { const int t = cmap[0]; cmap[0] = cmap[q]; cmap[q] = t; }
        __syncthreads();
    }
    pass(0, false);
    publish(0, n, 0, eb);
    if (!grid_barrier(bar, G, err)) return;

    for (int j = 0; j < n; ++j) {
        const int buf = j % 3;
        // (A) the sums of step j and row j, by position
        for (int c = j + tid; c < n; c += blockDim.x) {
            const int pc = cmap[c];
            const unsigned long long* src = lim + (size_t)buf * LS + (size_t)pc * 9;
            unsigned long long Lv[9];
#pragma unroll
            for (int u = 0; u < 9; ++u) Lv[u] = __ldcg(src + u);
            const dfl dr = qx_to_dfl(Lv, eb), di = qx_to_dfl(Lv + 3, eb), nn = qx_to_dfl(Lv + 6, eb);
            sD[c] = cdfl_pack({dr, di});
            sN[c] = make_float2(nn.hi, nn.lo);
            // row j; the pivot's entry from Pc (the previous pass kept that column there)
            sRow[c] = (c == j) ? __ldcg(Pc + (size_t)(j & 1) * N + j) : __ldcg(X + (int64_t)j * n + pc);
        }
        if (blockIdx.x == 0) {
            unsigned long long* z = lim + (size_t)((j + 2) % 3) * LS;
            for (size_t u = tid; u < LS; u += blockDim.x) z[u] = 0ull;
        }
        __syncthreads();
        // (B) reflector of the pivot column (one thread, double-float)
        const bool own_j = (j >= r0 && j < r1);
        if (tid == 0) {
            const dfl nrm2 = cdfl_unpack(sD[j]).re;      // sum |x_{i,p}|^2, i >= j (double-float)
            const cdfl xjj = cdfl_unpack(sRow[j]);
            cdfl alpha = cdfl_zero(), vj = cdfl_zero();
            dfl tau = {0.f, 0.f};
            if (nrm2.hi > 0.f) {
                const dfl a = dfl_sqrt(nrm2);
                const dfl ax2 = dfl_fma(xjj.re, xjj.re, dfl_mul(xjj.im, xjj.im));
                cdfl ph = {{1.f, 0.f}, {0.f, 0.f}};
                dfl ax = {0.f, 0.f};
                if (ax2.hi > 0.f) {
                    ax = dfl_sqrt(ax2);
                    const dfl rax = dfl_div(dfl{1.f, 0.f}, ax);
                    ph = {dfl_mul(xjj.re, rax), dfl_mul(xjj.im, rax)};
                }
                const dfl apx = dfl_add(a, ax);
                alpha = {dfl_neg(dfl_mul(ph.re, a)), dfl_neg(dfl_mul(ph.im, a))};
                vj = {dfl_mul(ph.re, apx), dfl_mul(ph.im, apx)};
                tau = dfl_div(dfl{1.f, 0.f}, dfl_mul(a, apx));
            }
            s_ref[0] = cdfl_pack(alpha);
            s_ref[1] = cdfl_pack(vj);
            s_tau = make_float2(tau.hi, tau.lo);
            if (own_j) R[j + (int64_t)cmap[j] * n] = cdfl_to(alpha);
        }
        __syncthreads();
        {
            // (C) w, row j of R, downdated norms
            const cdfl alpha = cdfl_unpack(s_ref[0]), vj = cdfl_unpack(s_ref[1]);
            const dfl tau = dfl_mk(s_tau);
            for (int c = j + 1 + tid; c < n; c += blockDim.x) {
                const cdfl d = cdfl_unpack(sD[c]), x = cdfl_unpack(sRow[c]);
                // d - conj(alpha) x
                const dfl tr = dfl_sub(d.re, dfl_fma(alpha.re, x.re, dfl_mul(alpha.im, x.im)));
                const dfl ti = dfl_sub(d.im, dfl_fma(alpha.re, x.im, dfl_neg(dfl_mul(alpha.im, x.re))));
                const cdfl wc = {dfl_mul(tau, tr), dfl_mul(tau, ti)};
                sW[c] = cdfl_pack(wc);
                // R_jc = x - vj wc
                const dfl rr = dfl_sub(x.re, dfl_fma(vj.re, wc.re, dfl_neg(dfl_mul(vj.im, wc.im))));
                const dfl ri = dfl_sub(x.im, dfl_fma(vj.re, wc.im, dfl_mul(vj.im, wc.re)));
                if (own_j) R[j + (int64_t)cmap[c] * n] = cmk(dfl_to(rr), dfl_to(ri));
                dfl nd = dfl_sub(dfl_mk(sN[c]), dfl_fma(rr, rr, dfl_mul(ri, ri)));
                if (nd.hi < 0.f) nd = {0.f, 0.f};
                sN[c] = make_float2(nd.hi, nd.lo);
            }
            __syncthreads();
            if (j + 1 < n) {
                const int q = pick(j + 1);
                if (tid == 0 && q < n && q != j + 1) {
                    // the next pivot moves to position j + 1; w is held by position, so it moves along
                    const int t = cmap[j + 1]; cmap[j + 1] = cmap[q]; cmap[q] = t;
                    const float4 tw = sW[j + 1]; sW[j + 1] = sW[q]; sW[q] = tw;
                }
                __syncthreads();
            }
        }
        if (j + 1 >= n) break;
        // (D) update this CTA's rows and accumulate the sums of step j + 1
        if (max(r0, (int64_t)(j + 1)) < r1) {
            pass(j + 1, true);
            publish(j + 1, n - j - 1, (j + 1) % 3, eb);
        }
        if (!grid_barrier(bar, G, err)) return;
    }
    if (blockIdx.x == 0)
        for (int c = tid; c < n; c += blockDim.x) perm[c] = cmap[c];
}

// R by position from R held by column (row j of column pc at Rc[j + pc n]), with the final
// permutation: R[j + c n] = Rc[j + perm[c] n] for c >= j, zero below the diagonal
__global__ void k_qr_place_R(const cplx* __restrict__ Rc, cplx* R, const int* __restrict__ perm, int n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int j = (int)(idx % n), c = (int)(idx / n);
    R[idx] = (c < j) ? cmk(0, 0) : Rc[j + (int64_t)perm[c] * n];
}

bem_status launch_house_qr(bem_ctx* h, cplx* X, int64_t N, int n, cplx* R, int* perm, bool dfl_arith) {
    if (n > 1024) return bem_fail(h, BEM_E_UNSUPPORTED, "QR: more than 1024 columns");
    if (N < n) return bem_fail(h, BEM_E_INVALID, "QR: fewer rows than columns");
    int nsm = 0;
    BEM_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const bool use_df = dfl_arith && n <= QR_NP;
    const int G = (int)std::min<int64_t>(nsm, (N + 15) / 16);
    bem_status st;
    if (use_df) {
        // X in place as double-float pairs (same 16 bytes per entry); three limb buffers
        // of 9 words per column and the window exponent, all starting at zero
        unsigned long long* lim = nullptr;
        const size_t lim_words = (size_t)3 * 9 * n + 1;
        float4* Pc = nullptr;                   // the next pivot column, two buffers
        // rows of R are written by column as the steps go (the pivots move columns between
        // positions after their earlier rows are known) and placed by position afterwards
        cplx* Rc = nullptr;
        cudaError_t ae = bem_dmalloc_async(h, (void**)&lim, sizeof(unsigned long long) * lim_words);
        if (ae == cudaSuccess) ae = bem_dmalloc_async(h, (void**)&Pc, sizeof(float4) * 2 * (size_t)N);
        if (ae == cudaSuccess) ae = bem_dmalloc_async(h, (void**)&Rc, sizeof(cplx) * (size_t)n * n);
        if (ae != cudaSuccess) {                // nothing launched yet: hand back what was taken
            bem_dfree_async(h, Rc);
            bem_dfree_async(h, Pc);
            bem_dfree_async(h, lim);
            return bem_cuda_check(h, ae, "QR temporaries");
        }
        BEM_CUDA(h, cudaMemsetAsync(lim, 0, sizeof(unsigned long long) * lim_words, h->stream));
        int* emax = reinterpret_cast<int*>(lim + 27 * (size_t)n);
        const int64_t cnt = N * (int64_t)n;
        BEM_TIMED(h, "k_to_dfl", (k_to_dfl<<<(unsigned)((cnt + 255) / 256), 256, 0, h->stream>>>(reinterpret_cast<float4*>(X), cnt)));
        BEM_LAUNCH(h, "k_to_dfl");
        float4* Xf = reinterpret_cast<float4*>(X);
        void* args_df[] = {&Xf, &N, &n, &Rc, &perm, &lim, &emax, &Pc, &h->bar, &h->dev_err};
        const size_t smem = (size_t)QR_NP * (8 * sizeof(float4) + 8 * sizeof(float) + 3 * sizeof(float4) + sizeof(float2));
        BEM_TIMED(h, "k_house_qr", st = coop_launch(h, (const void*)k_house_qr_df, G, QR_NT, args_df, "k_house_qr_df", smem));
        if (st == BEM_OK) {
            BEM_TIMED(h, "k_qr_place_R", (k_qr_place_R<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, h->stream>>>(Rc, R, perm, n)));
            BEM_LAUNCH(h, "k_qr_place_R");
        }
        bem_dfree_async(h, Rc);
        bem_dfree_async(h, lim);
        bem_dfree_async(h, Pc);
        return st;
    }
    double* partC = nullptr;
    cplx* partW = nullptr;
    unsigned long long* cnq = nullptr;
    cudaError_t ae = bem_dmalloc_async(h, (void**)&partC, sizeof(double) * (size_t)G * n);
    if (ae == cudaSuccess) ae = bem_dmalloc_async(h, (void**)&cnq, sizeof(unsigned long long) * 2 * (size_t)n);
    if (ae == cudaSuccess) ae = bem_dmalloc_async(h, (void**)&partW, sizeof(cplx) * (size_t)G * n);
    if (ae != cudaSuccess) {                    // nothing launched yet: hand back what was taken
        bem_dfree_async(h, partW);
        bem_dfree_async(h, cnq);
        bem_dfree_async(h, partC);
        return bem_cuda_check(h, ae, "QR temporaries");
    }
    BEM_CUDA(h, cudaMemsetAsync(cnq, 0, sizeof(unsigned long long) * 2 * (size_t)n, h->stream));
    void* args[] = {&X, &N, &n, &R, &perm, &partC, &cnq, &partW, &h->bar, &h->dev_err};
    BEM_TIMED(h, "k_house_qr", st = coop_launch(h, (const void*)k_house_qr, G, 256, args, "k_house_qr"));
    bem_dfree_async(h, partC);
    bem_dfree_async(h, cnq);
    bem_dfree_async(h, partW);
    return st;
}

// =========================================================================================
// One-sided Jacobi SVD of R (n x n, column-major): R V = U S.  Column pairs (p, q) of a
// round-robin tournament are rotated in parallel, one pair per CTA; rotation
//   R_p' = c R_p - s e^{-i phi} R_q,   R_q' = s e^{i phi} R_p + c R_q,
// where R_p^H R_q = |g| e^{i phi}, zeta = (b - a)/(2|g|), t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)),
// c = 1/sqrt(1+t^2), s = c t (a = |R_p|^2, b = |R_q|^2).
// =========================================================================================
__device__ __forceinline__ void tourney(int round, int idx, int np, int& p, int& q) {
    auto pos = [&](int k) { return (k == 0) ? 0 : ((round + k - 1) % (np - 1)) + 1; };
    p = pos(idx);
    q = pos(np - 1 - idx);
}

// Rotation of a column pair from A = |x|^2, B = |y|^2, G = x^H y (double-float sums), on
// values scaled by 2^-E with 2^E near max(A, B) (|G|^2 <= A B keeps everything below 1).
// Returns 0 for a converged pair (|G| <= 1e-14 |x| |y|), 1 for a rotation, 2 for a rotation
// with |G| > 1e-8 |x| |y| (a sweep with none of those is the last one: Jacobi's quadratic
// convergence leaves |G| near 1e-16 after it).  c, sem = s e^{-i phi}, sep = s e^{i phi}.
__device__ __forceinline__ int jac_rotation(const dfl sm[4], dfl& c, cdfl& sem, cdfl& sep) {
    const float mx = fmaxf(sm[0].hi, sm[1].hi);
    const float sc = (mx > 0.f) ? __int_as_float((254 - ((__float_as_int(mx) >> 23) & 255)) << 23) : 1.f;
    const dfl A = dfl_scale(sm[0], sc), Bv = dfl_scale(sm[1], sc);
    const dfl GR = dfl_scale(sm[2], sc), GI = dfl_scale(sm[3], sc);
    const dfl ag2 = dfl_fma(GR, GR, dfl_mul(GI, GI));
    const dfl ab = dfl_mul(A, Bv);
    if (!(ag2.hi > 0.f) || ag2.hi <= 1e-28f * ab.hi) return 0;
    const dfl rag = dfl_rsqrt(ag2);                       // 1/|g|
    const dfl zeta = dfl_scale(dfl_mul(dfl_sub(Bv, A), rag), 0.5f);
    dfl t;
    if (fabsf(zeta.hi) > 1e15f) {
        t = dfl_div(dfl{0.5f, 0.f}, zeta);               // 1/(2 zeta)
    } else {
        const dfl den = dfl_add(dfl{fabsf(zeta.hi), zeta.hi < 0.f ? -zeta.lo : zeta.lo},
                                dfl_sqrt(dfl_fma(zeta, zeta, dfl{1.f, 0.f})));
        t = dfl_div(dfl{zeta.hi >= 0.f ? 1.f : -1.f, 0.f}, den);
    }
    c = dfl_rsqrt(dfl_fma(t, t, dfl{1.f, 0.f}));
    const dfl sr = dfl_mul(dfl_mul(c, t), rag);
    const dfl srGR = dfl_mul(sr, GR), srGI = dfl_mul(sr, GI);
    sem = {srGR, dfl_neg(srGI)};
    sep = {srGR, srGI};
    return (ag2.hi > 1e-16f * ab.hi) ? 2 : 1;
}

// One-sided Jacobi on the columns of X (n x n, column-major).  Applied to X = R^H it
// leaves X_final = U Sigma with U the left singular vectors of R^H (= those of the block
// the QR came from); R^H from a QR is close to diagonally dominant, which makes the
// sweeps few.  128 threads per pair; one pair per CTA per round.
#define JAC_NT 128
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Rounds are ordered by data, not by grid barriers: every column carries a version (the
// rounds it has been through), a CTA starts its pair of round t of a sweep once both
// columns have reached version t, and publishes version t + 1 after writing them (release /
// acquire at GPU scope; column data bypass L1).  A CTA waits only on the two CTAs that
// last touched its columns, so consecutive rounds overlap across the grid.  One grid
// barrier per sweep decides convergence.  Waits are bounded (DEVERR_TIMEOUT).
// The columns are held in double-float (float4 per complex entry): dot products, their
// reductions and the rotation run on the FP32 pipe, the rotation scalars included (formed
// once per pair by one thread with double-float roots and quotients, which keeps the FP64
// pipe's long dependent latency off the round's critical path).
// EPT column entries per thread (n <= EPT JAC_NT).  The instance for n <= 256 is held to 85
// registers (six CTAs' worth per SM), so that one of its CTAs fits on an SM beside a CTA of
// the split-bf16 GEMM (320 threads x 168 registers) and the two can run at the same time.
template <int EPT>
__global__ void __launch_bounds__(JAC_NT, EPT <= 2 ? 6 : 1) k_jacobi(float4* X, int n, int* ver, int* flags, int max_sweeps,
                                                   unsigned* bar, int* err) {
    __shared__ float2 red[JAC_NT / 32][4];
    __shared__ int s_ok;
    const unsigned G = gridDim.x;
    const int np = n + (n & 1);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int round = 0; round < np - 1; ++round) {
            const int target = sweep * (np - 1) + round;
            for (int idx = blockIdx.x; idx < np / 2; idx += G) {
                int p, q;
                tourney(round, idx, np, p, q);
                if (p > q) { int t = p; p = q; q = t; }
                if (tid == 0) {
                    // wait for one column's version, then the other's: one acquire load per
                    // poll (an acquire orders the loads after it, so two per poll would run
                    // one after the other)
                    int ok = 1;
                    bool rp = (p >= n);
                    for (long long spins = 0;; ++spins) {
                        if (!rp) rp = ld_acquire(ver + p) >= target;
                        if (rp && ((q >= n) || ld_acquire(ver + q) >= target)) break;
                        if (spins > (1ll << 24)) { atomicOr(err, DEVERR_TIMEOUT); ok = 0; break; }
                        if ((spins & 255) == 255 && *(volatile int*)err) { ok = 0; break; }
                        if (spins > 32) __nanosleep(32);
                    }
                    s_ok = ok;
                }
                __syncthreads();
                if (!s_ok) return;
                if (q < n) {       // both columns real (p < q)
                    float4* Xp = X + (int64_t)p * n;
                    float4* Xq = X + (int64_t)q * n;
                    cdfl x[EPT], y[EPT];
                    dfl a = {0.f, 0.f}, b = {0.f, 0.f}, gr = {0.f, 0.f}, gi = {0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        const int i = tid + JAC_NT * e;
                        x[e] = (i < n) ? cdfl_unpack(__ldcg(Xp + i)) : cdfl_zero();
                        y[e] = (i < n) ? cdfl_unpack(__ldcg(Xq + i)) : cdfl_zero();
                        if (i < n) {
                            a = dfl_fma(x[e].im, x[e].im, dfl_fma(x[e].re, x[e].re, a));
                            b = dfl_fma(y[e].im, y[e].im, dfl_fma(y[e].re, y[e].re, b));
                            gr = dfl_fma(x[e].im, y[e].im, dfl_fma(x[e].re, y[e].re, gr));          // conj(x) y
                            gi = dfl_fma(dfl_neg(x[e].im), y[e].re, dfl_fma(x[e].re, y[e].im, gi));
                        }
                    }
                    dfl v4[4] = {a, b, gr, gi};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        for (int o = 16; o > 0; o >>= 1) {
                            const dfl t = {__shfl_xor_sync(0xffffffffu, v4[k].hi, o),
                                           __shfl_xor_sync(0xffffffffu, v4[k].lo, o)};
                            v4[k] = dfl_add(v4[k], t);
                        }
                    if (lane == 0)
                        for (int k = 0; k < 4; ++k) red[wid][k] = make_float2(v4[k].hi, v4[k].lo);
                    __syncthreads();
                    // every thread sums the warps' partials in the same order and forms the
                    // same rotation (no second barrier, no broadcast)
                    dfl sm[4];
                    for (int k = 0; k < 4; ++k) {
                        dfl t = dfl_mk(red[0][k]);
                        for (int w = 1; w < JAC_NT / 32; ++w) t = dfl_add(t, dfl_mk(red[w][k]));
                        sm[k] = t;
                    }
                    dfl c;
                    cdfl sem, sep;
                    const int rot = jac_rotation(sm, c, sem, sep);
                    if (rot == 2 && tid == 0) flags[sweep] = 1;
                    if (rot) {
#pragma unroll
                        for (int e = 0; e < EPT; ++e) {
                            const int i = tid + JAC_NT * e;
                            if (i >= n) continue;
                            // x' = c x - sem y ;  y' = sep x + c y
                            cdfl xn, yn;
                            xn.re = dfl_fma(dfl_neg(sem.re), y[e].re, dfl_fma(sem.im, y[e].im, dfl_mul(c, x[e].re)));
                            xn.im = dfl_fma(dfl_neg(sem.re), y[e].im, dfl_fma(dfl_neg(sem.im), y[e].re, dfl_mul(c, x[e].im)));
                            yn.re = dfl_fma(sep.re, x[e].re, dfl_fma(dfl_neg(sep.im), x[e].im, dfl_mul(c, y[e].re)));
                            yn.im = dfl_fma(sep.re, x[e].im, dfl_fma(sep.im, x[e].re, dfl_mul(c, y[e].im)));
                            __stcg(Xp + i, cdfl_pack(xn));
                            __stcg(Xq + i, cdfl_pack(yn));
                        }
                    }
                }
                __syncthreads();              // the pair's stores precede its release
                if (tid == 0) {
                    // one release fence orders the CTA's stores (made cumulative by the barrier
                    // above) before both versions; a second st.release would wait for the first
                    __threadfence();
                    if (p < n) st_relaxed(ver + p, target + 1);
                    if (q < n) st_relaxed(ver + q, target + 1);
                }
            }
        }
        if (!grid_barrier(bar, G, err)) return;
        if (*(volatile int*)(flags + sweep) == 0) return;
    }
}

// sigma_c = |X_c| (X in double-float), sorted descending; E[:, rank] = X_c / sigma_c (a
// unit vector e_c when sigma_c = 0, which is then below any truncation threshold), with its
// rows put back in the original order when the QR pivoted (E[perm[i], rank] = X[i, c];
// perm may be null)
__global__ void k_sort_sv(const float4* X, int n, const int* perm, double* sigma, cplx* E, double* tmp) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const cdfl x = cdfl_unpack(X[(int64_t)c * n + i]);
            const double re = dfl_to(x.re), im = dfl_to(x.im);
            s += re * re + im * im;
        }
        tmp[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double sc = tmp[c];
        int rank = 0;
        for (int d = 0; d < n; ++d) {
            const double sd = tmp[d];
            if (sd > sc || (sd == sc && d < c)) ++rank;
        }
        sigma[rank] = sc;
        const double inv = (sc > 0.0) ? 1.0 / sc : 0.0;
        for (int i = 0; i < n; ++i) {
            const cdfl x = cdfl_unpack(X[(int64_t)c * n + i]);
            E[(int64_t)rank * n + (perm ? perm[i] : i)] =
                (sc > 0.0) ? cmk(dfl_to(x.re) * inv, dfl_to(x.im) * inv) : cmk(i == c ? 1.0 : 0.0, 0.0);
        }
    }
}

// X = R^H (n x n) in double-float
__global__ void k_conj_transpose(const cplx* R, float4* X, int n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int64_t i = idx % n, j = idx / n;
    const cplx v = R[j + i * n];
    X[idx] = cdfl_pack({dfl_from(v.x), dfl_from(-v.y)});
}

// scratch of launch_jacobi_svd: X (n x n double-float), the sweep flags, the column
// versions and the norms, each 256-byte aligned
#define JAC_MAX_SWEEPS 40
static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
size_t jacobi_scratch_bytes(int n) {
    return al256(sizeof(float4) * (size_t)n * n) + al256(sizeof(int) * JAC_MAX_SWEEPS) + al256(sizeof(int) * (size_t)n) +
           al256(sizeof(double) * (size_t)n);
}

// scratch: jacobi_scratch_bytes(n) bytes the caller keeps until the stream has run the SVD
// (the handle's workspace: no stream-ordered allocation, so the SVD can run on any stream)
bem_status launch_jacobi_svd(bem_ctx* h, cplx* R, int n, const int* perm, double* sigma, cplx* E, void* scratch) {
    if (n > 1024) return bem_fail(h, BEM_E_UNSUPPORTED, "Jacobi SVD: more than 1024 columns");
    const int max_sweeps = JAC_MAX_SWEEPS;
    char* sp = (char*)scratch;
    float4* X = (float4*)sp;
    sp += al256(sizeof(float4) * (size_t)n * n);
    int* flags = (int*)sp;
    sp += al256(sizeof(int) * max_sweeps);
    int* ver = (int*)sp;
    sp += al256(sizeof(int) * (size_t)n);
    double* tmp = (double*)sp;
    BEM_CUDA(h, cudaMemsetAsync(ver, 0, sizeof(int) * n, h->stream));
    BEM_CUDA(h, cudaMemsetAsync(flags, 0, sizeof(int) * max_sweeps, h->stream));
    BEM_TIMED(h, "k_conj_transpose",
              (k_conj_transpose<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, h->stream>>>(R, X, n)));
    BEM_LAUNCH(h, "k_conj_transpose");
    int ms = max_sweeps;
    void* args[] = {&X, &n, &ver, &flags, &ms, &h->bar, &h->dev_err};
    bem_status st;
    const void* jk = (n <= 2 * JAC_NT) ? (const void*)k_jacobi<2>
                     : (n <= 4 * JAC_NT) ? (const void*)k_jacobi<4> : (const void*)k_jacobi<8>;
    BEM_TIMED(h, "k_jacobi", st = coop_launch(h, jk, (n + 1) / 2, JAC_NT, args, "k_jacobi"));
    if (st == BEM_OK) {
        BEM_TIMED(h, "k_sort_sv", (k_sort_sv<<<1, 256, 0, h->stream>>>(X, n, perm, sigma, E, tmp)));
        BEM_LAUNCH(h, "k_sort_sv");
    }
    return st;
}

// =========================================================================================
// Gauss-Jordan inversion with partial pivoting of A (r x r) on the augmented [A | I]
// (r x 2r, column-major, ld = r).  CTA b owns a block of augmented columns.  Step j needs
// only the pivot column j as left by step j - 1: its owner publishes that copy in a buffer
// of its own (colbuf + j r, all r kept, so no copy is ever overwritten) and then a flag
// (release); every CTA waits for that flag alone (acquire, bounded), finds the pivot and
// updates its columns, the owner of column j + 1 first.  Steps chain through the pivot
// columns instead of grid barriers, so a CTA runs ahead as far as the pivots allow.
// =========================================================================================
__global__ void __launch_bounds__(256) k_gauss_jordan(cplx* M, int r, cplx* colbuf, int* ready, int* err) {
    extern __shared__ cplx colj[];
    __shared__ double wv[8];
    __shared__ int wi[8];
    __shared__ int s_ok;
    const unsigned G = gridDim.x;
    const int ncol = 2 * r;
    const int cb = (ncol + G - 1) / G;
    const int c0 = blockIdx.x * cb, c1 = min(ncol, c0 + cb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < r; ++j) {
        if (threadIdx.x == 0) {
            int ok = 1;
            for (long long spins = 0; ld_acquire(ready + j) == 0; ++spins) {
                if (spins > (1ll << 24)) { atomicOr(err, DEVERR_TIMEOUT); ok = 0; break; }
                if ((spins & 255) == 255 && *(volatile int*)err) { ok = 0; break; }
                if (spins > 32) __nanosleep(32);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        // pivot column j as left by step j - 1
        const cplx* buf = colbuf + (size_t)j * r;
        for (int i = threadIdx.x; i < r; i += blockDim.x) colj[i] = __ldcg(buf + i);
        __syncthreads();
        // argmax |colj[i]|, i >= j (ties to the lower row)
        double best = -1.0;
        int bi = r;
        for (int i = j + threadIdx.x; i < r; i += blockDim.x) {
            const double v = cabs2(colj[i]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { wv[wid] = best; wi[wid] = bi; }
        __syncthreads();
        double bb = wv[0];
        int p = wi[0];
        for (int q = 1; q < nw; ++q)
            if (wv[q] > bb || (wv[q] == bb && wi[q] < p)) { bb = wv[q]; p = wi[q]; }
        if (!(bb > 0.0) || p >= r) {
            if (threadIdx.x == 0) atomicOr(err, DEVERR_SINGULAR);
            p = j;
        }
        const cplx cj = colj[j], cp = colj[p];
        __syncthreads();
        if (threadIdx.x == 0 && p != j) { colj[j] = cp; colj[p] = cj; }
        __syncthreads();
        const cplx pv = colj[j];
        const bool sing = !(cabs2(pv) > 0.0);
        const cplx ipv = sing ? cmk(0, 0) : cdiv(cmk(1, 0), pv);
        // this CTA's columns c >= j (eliminated ones stay unit columns), column j + 1 first
        const int lo = max(c0, j);
        const int first = (j + 1 >= lo && j + 1 < c1) ? j + 1 : -1;
        const int cnt = c1 - lo;
        for (int t = wid; t < cnt; t += nw) {
            int c;
            if (first < 0) c = lo + t;
            else c = (t == 0) ? first : ((lo + t - 1 >= first) ? lo + t : lo + t - 1);
            cplx* col = M + (int64_t)c * r;
            // swap rows j, p of this column and normalise row j
            const cplx xj = cmul(col[p], ipv), xp = col[j];
            __syncwarp();
            cplx* nxt = (c == j + 1 && j + 1 < r) ? colbuf + (size_t)(j + 1) * r : nullptr;
            for (int i = lane; i < r; i += 32) {
                cplx v;
                if (i == j) v = xj;
                else v = csub((i == p) ? xp : col[i], cmul(colj[i], xj));
                col[i] = v;
                if (nxt) __stcg(nxt + i, v);
            }
            __syncwarp();
            if (nxt && lane == 0) {
                // the warp's copy before the flag: one fence, made cumulative by the warp barrier
                __threadfence();
                st_relaxed(ready + j + 1, 1);
            }
        }
        // (the next step reloads colj only after its first barrier, which every warp of this
        // step reaches after its updates)
    }
}

__global__ void k_augment(const cplx* K, cplx* M, cplx* colbuf, int* ready, int r) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)r * 2 * r) return;
    const int64_t i = idx % r, c = idx / r;
    M[idx] = (c < r) ? K[i + c * r] : cmk((c - r) == i ? 1.0 : 0.0, 0.0);
    if (c == 0) colbuf[i] = K[i];
    if (c < r && i == 0) ready[c] = (c == 0) ? 1 : 0;   // step 0's pivot column is K's first
}

// scratch of launch_gauss_jordan: [K | I] (r x 2r), the published pivot columns (r x r) and
// their flags, each 256-byte aligned
size_t gauss_jordan_scratch_bytes(int r) {
    return al256(sizeof(cplx) * (size_t)r * 2 * r) + al256(sizeof(cplx) * (size_t)r * r) + al256(sizeof(int) * (size_t)r);
}

// scratch: gauss_jordan_scratch_bytes(r) bytes, as for launch_jacobi_svd
bem_status launch_gauss_jordan(bem_ctx* h, const cplx* K, cplx* Kinv, int r, void* scratch) {
    char* sp = (char*)scratch;
    cplx* M = (cplx*)sp;
    sp += al256(sizeof(cplx) * (size_t)r * 2 * r);
    cplx* colbuf = (cplx*)sp;
    sp += al256(sizeof(cplx) * (size_t)r * r);
    int* ready = (int*)sp;
    BEM_TIMED(h, "k_augment", (k_augment<<<(unsigned)(((int64_t)r * 2 * r + 255) / 256), 256, 0, h->stream>>>(K, M, colbuf, ready, r)));
    BEM_LAUNCH(h, "k_augment");
    const size_t smem = sizeof(cplx) * (size_t)r;
    if (smem > 48 * 1024)
        BEM_CUDA(h, cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nsm = 0, per = 0;
    BEM_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    BEM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gauss_jordan, 256, smem));
    if (per < 1) return bem_fail(h, BEM_E_CUDA, "k_gauss_jordan cannot be resident");
    // three augmented columns per CTA: the per-step FP64 update spreads over about 2r/3 SMs
    int G = std::min(nsm * per, std::max(1, (2 * r + 2) / 3));
    void* args[] = {&M, &r, &colbuf, &ready, &h->dev_err};
    cudaError_t lerr;
    BEM_TIMED(h, "k_gauss_jordan",
              lerr = cudaLaunchCooperativeKernel((const void*)k_gauss_jordan, dim3(G), dim3(256), args, smem, h->stream));
    BEM_CUDA(h, lerr);
    BEM_LAUNCH(h, "k_gauss_jordan");
    BEM_CUDA(h, cudaMemcpy2DAsync(Kinv, sizeof(cplx) * r, M + (size_t)r * r, sizeof(cplx) * r,
                                  sizeof(cplx) * r, r, cudaMemcpyDeviceToDevice, h->stream));
    return BEM_OK;
}

// =========================================================================================
// small elementwise helpers
// =========================================================================================
// out[i] = in[i] + shift
__global__ void k_shift(const double* in, double* out, int64_t n, double shift) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] + shift;
}
bem_status launch_shift(bem_ctx* h, const double* in, double* out, int64_t n, double shift) {
    BEM_TIMED(h, "k_shift", (k_shift<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(in, out, n, shift)));
    BEM_LAUNCH(h, "k_shift");
    return BEM_OK;
}
// x[:, j] *= s[j] (complex column scale)
__global__ void k_scale_cols(cplx* x, int64_t ldx, const cplx* s, int64_t rows, int64_t cols) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    x[i + j * ldx] = cmul(x[i + j * ldx], s[j]);
}
bem_status launch_scale_cols(bem_ctx* h, cplx* x, int64_t ldx, const cplx* s, int64_t rows, int64_t cols) {
    const int64_t n = rows * cols;
    BEM_TIMED(h, "k_scale_cols", (k_scale_cols<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(x, ldx, s, rows, cols)));
    BEM_LAUNCH(h, "k_scale_cols");
    return BEM_OK;
}
// y = a * conj(x) over a rows x cols block (leading dimensions ldx, ldy)
__global__ void k_conj_scale(const cplx* x, int64_t ldx, cplx* y, int64_t ldy, cplx a, int64_t rows, int64_t cols) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    y[i + j * ldy] = cmul(a, cconj(x[i + j * ldx]));
}
bem_status launch_conj_scale(bem_ctx* h, const cplx* x, int64_t ldx, cplx* y, int64_t ldy, cplx a, int64_t rows,
                             int64_t cols) {
    const int64_t n = rows * cols;
    BEM_TIMED(h, "k_conj_scale", (k_conj_scale<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(x, ldx, y, ldy, a, rows, cols)));
    BEM_LAUNCH(h, "k_conj_scale");
    return BEM_OK;
}
__global__ void k_axpby(cplx* y, int64_t ldy, const cplx* x, int64_t ldx, cplx a, cplx b, int64_t rows, int64_t cols) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t rr = idx % rows, cc = idx / rows;
    const cplx xv = x[rr + cc * ldx];
    cplx v = cmul(a, xv);
    if (b.x != 0.0 || b.y != 0.0) v = cadd(v, cmul(b, y[rr + cc * ldy]));
    y[rr + cc * ldy] = v;
}
// y = a x + b y with real a, b: a 2D grid (no index division) and two FP64 operations per
// component, which keeps it at the memory rate (complex coefficients cost the FP64 pipe)
__global__ void k_axpby_real(cplx* y, int64_t ldy, const cplx* x, int64_t ldx, double a, double b, int64_t rows,
                             int64_t cols) {
    const int64_t rr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rr >= rows) return;
    for (int64_t cc = blockIdx.y; cc < cols; cc += gridDim.y) {
        const cplx xv = x[rr + cc * ldx];
        cplx v = cmk(a * xv.x, a * xv.y);
        if (b != 0.0) {
            const cplx yv = y[rr + cc * ldy];
            v = cmk(fma(b, yv.x, v.x), fma(b, yv.y, v.y));
        }
        y[rr + cc * ldy] = v;
    }
}
bem_status launch_axpby(bem_ctx* h, cplx* y, int64_t ldy, const cplx* x, int64_t ldx, cplx a, cplx b,
                        int64_t rows, int64_t cols) {
    const int64_t tot = rows * cols;
    if (tot == 0) return BEM_OK;
    if (a.y == 0.0 && b.y == 0.0) {
        dim3 grid((unsigned)((rows + 255) / 256), (unsigned)std::min<int64_t>(cols, 65535));
        BEM_TIMED(h, "k_axpby", (k_axpby_real<<<grid, 256, 0, h->stream>>>(y, ldy, x, ldx, a.x, b.x, rows, cols)));
    } else {
        BEM_TIMED(h, "k_axpby", (k_axpby<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(y, ldy, x, ldx, a, b, rows, cols)));
    }
    BEM_LAUNCH(h, "k_axpby");
    return BEM_OK;
}

__global__ void k_add_identity(cplx* A, int64_t ld, int r, cplx d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    A[i + i * ld] = cadd(A[i + i * ld], d);
}
bem_status launch_add_identity(bem_ctx* h, cplx* A, int64_t ld, int r, cplx d) {
    BEM_TIMED(h, "k_add_identity", (k_add_identity<<<(r + 255) / 256, 256, 0, h->stream>>>(A, ld, r, d)));
    BEM_LAUNCH(h, "k_add_identity");
    return BEM_OK;
}

// double -> float from the bit fields, significand truncated (a norm estimate needs no
// more; FP64 conversions and squares would run on the slow FP64 pipe); values outside
// the float range saturate or flush
__device__ __forceinline__ float d2f_trunc(double v) {
    const long long b = __double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    if (E <= 0) return 0.f;
    const unsigned sgn = (unsigned)((unsigned long long)b >> 63) << 31;
    if (E >= 255) return __uint_as_float(sgn | 0x7F7FFFFFu);
    return __uint_as_float(sgn | ((unsigned)E << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
}
// out_max = max over columns of |num_c| / |den_c| (2-norms, FP32 accumulation: the ratio
// is a convergence test, far looser than FP32's precision); one CTA per column, then max
__global__ void k_col_ratio(const cplx* num, int64_t ldn, const cplx* den, int64_t ldd, int64_t rows, double* ratios) {
    __shared__ float red[2][32];
    const int64_t c = blockIdx.x;
    float a = 0.f, b = 0.f;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
        const cplx u = num[i + c * ldn], w = den[i + c * ldd];
        const float ur = d2f_trunc(u.x), ui = d2f_trunc(u.y), wr = d2f_trunc(w.x), wi = d2f_trunc(w.y);
        a = fmaf(ur, ur, fmaf(ui, ui, a));
        b = fmaf(wr, wr, fmaf(wi, wi, b));
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = a; red[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { A += red[0][q]; B += red[1][q]; }
        ratios[c] = (B > 0.0) ? sqrt(A / B) : sqrt(A);
    }
}
__global__ void k_max(const double* v, int64_t n, double* out) {
    __shared__ double red[32];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, red[q]);
        *out = r;
    }
}
bem_status launch_col_norm_ratio(bem_ctx* h, const cplx* num, int64_t ldn, const cplx* den, int64_t ldd,
                                 int64_t rows, int64_t cols, double* out_max) {
    double* ratios = nullptr;
    BEM_CUDA(h, bem_dmalloc_async(h, (void**)&ratios, sizeof(double) * cols));
    BEM_TIMED(h, "k_col_ratio", (k_col_ratio<<<(unsigned)cols, 256, 0, h->stream>>>(num, ldn, den, ldd, rows, ratios)));
    BEM_LAUNCH(h, "k_col_ratio");
    BEM_TIMED(h, "k_max", (k_max<<<1, 256, 0, h->stream>>>(ratios, cols, out_max)));
    BEM_LAUNCH(h, "k_max");
    bem_dfree_async(h, ratios);
    return BEM_OK;
}

bem_status launch_copy2d(bem_ctx* h, void* dst, int64_t ldd, const void* src, int64_t lds, int64_t rows,
                         int64_t cols, size_t elem) {
    BEM_CUDA(h, cudaMemcpy2DAsync(dst, elem * ldd, src, elem * lds, elem * rows, cols,
                                  cudaMemcpyDeviceToDevice, h->stream));
    return BEM_OK;
}

// =========================================================================================
// Constant-vector correction of the filtered product.  N's row sums are O(k^2) of its
// entries (Maue's form: the derivative term's row sums vanish), so at low k the product
// P = Y N loses B's action on the constant vector 1 to rounding -- that of the split
// products, relative to the entries, and that of N's stored entries, up to
// 2^-53 sum_j |N_ij| per row -- while that action carries the Calderon product's smallest
// eigenvalue.  With w = N 1 (the exact row sums the assembly accumulates from N's k^2
// term, or else summed in FP64 from the stored N) the product is corrected along 1 only:
//     P <- P + (Y w - P 1) 1^T / N      (P's action on the complement of 1 is unchanged).
// =========================================================================================
__device__ __forceinline__ cplx block_csum(cplx v, double* red) {
    return cmk(block_sum(v.x, red), block_sum(v.y, red));
}

// w[j] = sum_i A[i + j lda], one CTA per column (A = N is complex symmetric: w = N 1)
__global__ void __launch_bounds__(256) k_col_sums(const cplx* __restrict__ A, int64_t lda, int64_t rows, cplx* w) {
    __shared__ double red[32];
    const int64_t j = blockIdx.x;
    cplx acc = cmk(0, 0);
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) acc = cadd(acc, A[i + j * lda]);
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) w[j] = acc;
}

// c_i = (sum_j Y[i + j ld] w_j - sum_j P[i + j ld]) / N, one CTA per row i
__global__ void __launch_bounds__(256) k_const_defect(const cplx* __restrict__ Y, const cplx* __restrict__ P,
                                                      int64_t ld, int64_t N, const cplx* __restrict__ w, cplx* c) {
    __shared__ double red[32];
    const int64_t i = blockIdx.x;
    cplx t = cmk(0, 0), s = cmk(0, 0);
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        t = cadd(t, cmul(Y[i + j * ld], w[j]));
        s = cadd(s, P[i + j * ld]);
    }
    t = block_csum(t, red);
    s = block_csum(s, red);
    if (threadIdx.x == 0) c[i] = cscale(csub(t, s), 1.0 / (double)N);
}

// P[i + j ld] += c_i
__global__ void k_add_row_const(cplx* P, int64_t ld, int64_t rows, int64_t N, const cplx* __restrict__ c) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * N) return;
    const int64_t i = idx % rows, j = idx / rows;
    P[i + j * ld] = cadd(P[i + j * ld], c[i]);
}

bem_status launch_const_correction(bem_ctx* h, const cplx* Wm, const cplx* w1, const cplx* Y, cplx* P, int64_t nc,
                                   int64_t N, cplx* scratch) {
    cplx* w = scratch;              // N
    cplx* c = scratch + N;          // nc
    if (w1) {
        w = const_cast<cplx*>(w1);
    } else {
        BEM_TIMED(h, "k_col_sums", (k_col_sums<<<(unsigned)N, 256, 0, h->stream>>>(Wm, N, N, w)));
        BEM_LAUNCH(h, "k_col_sums");
    }
    BEM_TIMED(h, "k_const_defect", (k_const_defect<<<(unsigned)nc, 256, 0, h->stream>>>(Y, P, nc, N, w, c)));
    BEM_LAUNCH(h, "k_const_defect");
    BEM_TIMED(h, "k_add_row_const", (k_add_row_const<<<(unsigned)((nc * N + 255) / 256), 256, 0, h->stream>>>(P, nc, nc, N, c)));
    BEM_LAUNCH(h, "k_add_row_const");
    return BEM_OK;
}

// =========================================================================================
// Differentiation helpers: amplitude gradient and the chain to curve coefficients
// =========================================================================================
// g[w] = sum_i conj(v[i + w ldv]) lam[i + w ldl], one CTA per column (fixed-order reduction)
__global__ void __launch_bounds__(256) k_col_cdot(const cplx* __restrict__ v, int64_t ldv, const cplx* __restrict__ lam,
                                                  int64_t ldl, int64_t rows, cplx* g) {
    __shared__ double red[32];
    const int64_t w = blockIdx.x;
    cplx acc = cmk(0, 0);
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) acc = cadd(acc, cmul(cconj(v[i + w * ldv]), lam[i + w * ldl]));
    acc = block_csum(acc, red);
    if (threadIdx.x == 0) g[w] = acc;
}
bem_status launch_col_cdot(bem_ctx* h, const cplx* v, int64_t ldv, const cplx* lam, int64_t ldl, int64_t rows,
                           int64_t cols, cplx* g) {
    BEM_TIMED(h, "k_col_cdot", (k_col_cdot<<<(unsigned)cols, 256, 0, h->stream>>>(v, ldv, lam, ldl, rows, g)));
    BEM_LAUNCH(h, "k_col_cdot");
    return BEM_OK;
}

// out[p] = sum_j T[p n + j] x[j] (T: P x n row-major, one CTA per p)
__global__ void __launch_bounds__(256) k_row_dot(const double* __restrict__ T, int64_t n, const double* __restrict__ x,
                                                 double* out) {
    __shared__ double red[32];
    const int64_t p = blockIdx.x;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) acc += T[p * n + j] * x[j];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[p] = acc;
}
bem_status launch_row_dot(bem_ctx* h, const double* T, int64_t P, int64_t n, const double* x, double* out) {
    BEM_TIMED(h, "k_row_dot", (k_row_dot<<<(unsigned)P, 256, 0, h->stream>>>(T, n, x, out)));
    BEM_LAUNCH(h, "k_row_dot");
    return BEM_OK;
}
