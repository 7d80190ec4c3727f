// Host-side launchers shared between the CUDA translation units (internal).
#pragma once

#include "common.cuh"

#define BEM_SERIES_MAX 24
// Entries of N with cyclic |i - j| <= TC_W_BAND (capped at (N - 1)/2) are applied in
// double-float next to the split-bf16 product of the rest
#define TC_W_BAND 64

// Small-argument expansions in r of the kernels (coefficients depend on k only):
//   g2(r)                    = sum_m r^{2m} (A_m + B_m ln r)
//   -(i k/4) H1^(1)(k r) / r = -1/(2 pi r^2) + sum_m r^{2m} (E_m + F_m ln r)
struct SeriesCoef {
    int nm;
    double2 A[BEM_SERIES_MAX];
    double B[BEM_SERIES_MAX];
    double2 E[BEM_SERIES_MAX];
    double F[BEM_SERIES_MAX];
};

void series_coefficients(double k, double hmax, SeriesCoef* sc);
cudaError_t init_gauss_tables();

// assemble.cu
bem_status launch_geometry(bem_ctx* h, const double* verts, int64_t N, double* stats_dev);
bem_status launch_assemble(bem_ctx* h, unsigned ops);
// S and N of nprob prepared handles in one persistent launch (global tile queue) on hs[0]'s stream
bem_status launch_assemble_batch(bem_ctx** hs, int nprob);
bem_status launch_rhs(bem_ctx* h, const double* angles, int64_t nrhs, cplx* f, cplx* hz, int64_t ld);
// line sources at src (2 nsrc doubles, (x, y) pairs): f = -<phi, d g2(|x - r0|)/d nu>, hz = <phi, g2>
bem_status launch_rhs_point(bem_ctx* h, const double* src, int64_t nsrc, cplx* f, cplx* hz, int64_t ld);
// shape gradient: d/dverts Re sum(Omega^S .* S + Omega^W .* N) (Omega passed transposed),
// d/dverts Re sum om .* f(angles), and the Gram terms of four signed (P, Q) block pairs
bem_status launch_assemble_vjp(bem_ctx* h, const cplx* OmS_T, const cplx* OmW_T, double* grad);
bem_status launch_rhs_vjp(bem_ctx* h, const double* angles, int64_t nang, const cplx* om, int64_t ld, double* grad);
bem_status launch_gram_vjp(bem_ctx* h, int nrhs, const cplx* const* P_dev, const cplx* const* Q_dev,
                           const double* sign_dev, double* grad);

// linalg.cu
enum { OP_N = 0, OP_T = 1, OP_C = 2 };
// C = A B in double-float (complex FP64 storage, no transposes, alpha = 1, beta = 0)
bem_status zgemm_df(bem_ctx* h, int64_t M, int64_t Nc, int64_t K, const cplx* A, int64_t lda, const cplx* B,
                    int64_t ldb, cplx* C, int64_t ldc);
bem_status zgemm(bem_ctx* h, int opa, int opb, int64_t M, int64_t Nc, int64_t K, cplx alpha,
                 const cplx* A, int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc);
bem_status dzgemm_realA(bem_ctx* h, int opa, int64_t M, int64_t Nc, int64_t K, double alpha,
                        const double* A, int64_t lda, const cplx* B, int64_t ldb, double beta,
                        cplx* C, int64_t ldc);
// G^-1 (mode 0) or F^-T = (I + r Z)^-1 * sqrt(6 r/h) (mode 1) along index i of a strided array
// (equal-chord meshes; on a general mesh the bordered factor of mesh.cu, G = F^T F)
bem_status apply_gram_inverse(bem_ctx* h, int mode, const cplx* in, cplx* out, cplx* tmp,
                              int64_t N, int64_t ncols, int64_t si, int64_t sc, double hbar,
                              bool conj_out);
bem_status launch_fourier_basis(bem_ctx* h, double* Q, int64_t N, int64_t ncols, int include_kernel,
                                double* gm, double hbar);
bem_status launch_finish_B(bem_ctx* h, cplx* B, const double* gm, const double* Q, int64_t ncols,
                           int64_t N);
bem_status launch_row_scale(bem_ctx* h, const cplx* in, cplx* out, const double* s, int pw,
                            int64_t rows, int64_t cols, int64_t ld);
bem_status launch_scale_real_cols(bem_ctx* h, const double* in, double* out, const double* s, int pw,
                                  int64_t rows, int64_t cols);
// dfl_arith: double-float arithmetic on the FP32 pipe (X is overwritten in that format)
bem_status launch_house_qr(bem_ctx* h, cplx* X, int64_t N, int n, cplx* R, int* perm, bool dfl_arith);
size_t jacobi_scratch_bytes(int n);
bem_status launch_jacobi_svd(bem_ctx* h, cplx* R, int n, const int* perm, double* sigma, cplx* E, void* scratch);
size_t gauss_jordan_scratch_bytes(int r);
bem_status launch_gauss_jordan(bem_ctx* h, const cplx* K, cplx* Kinv, int r, void* scratch);
bem_status launch_axpby(bem_ctx* h, cplx* y, int64_t ldy, const cplx* x, int64_t ldx, cplx a, cplx b,
                        int64_t rows, int64_t cols);   // y = a*x + b*y
bem_status launch_add_identity(bem_ctx* h, cplx* A, int64_t ld, int r, cplx d);
bem_status launch_col_norm_ratio(bem_ctx* h, const cplx* num, int64_t ldn, const cplx* den,
                                 int64_t ldd, int64_t rows, int64_t cols, double* out_max);
bem_status launch_scale_cols(bem_ctx* h, cplx* x, int64_t ldx, const cplx* s, int64_t rows, int64_t cols);
bem_status launch_shift(bem_ctx* h, const double* in, double* out, int64_t n, double shift);
bem_status launch_conj_scale(bem_ctx* h, const cplx* x, int64_t ldx, cplx* y, int64_t ldy, cplx a, int64_t rows,
                             int64_t cols);   // y = a conj(x)
// P <- P + (Y w - P 1) 1^T / N for the n x N product P = Y W (ld = nc), w = W 1 given (w1) or
// summed from W; scratch: N + nc
bem_status launch_const_correction(bem_ctx* h, const cplx* Wm, const cplx* w1, const cplx* Y, cplx* P, int64_t nc,
                                   int64_t N, cplx* scratch);
// g[w] = v[:, w]^H lam[:, w]
bem_status launch_col_cdot(bem_ctx* h, const cplx* v, int64_t ldv, const cplx* lam, int64_t ldl, int64_t rows,
                           int64_t cols, cplx* g);
// out = T x for T: P x n row-major (FP64)
bem_status launch_row_dot(bem_ctx* h, const double* T, int64_t P, int64_t n, const double* x, double* out);
// mesh.cu (non-equal-chord meshes)
// bordered LDL^T of cL L + cG G (4N doubles at fac) on h's stream
bem_status launch_cyc_factor(bem_ctx* h, double cL, double cG, double* fac);
// apply_gram_inverse for a general mesh: mode 0 G^-1, mode 1 D^-1/2 L^-1 (rows times F^-1)
// (chunked over N; tmp holds tmp_elems >= 5 ceil((N-2)/64) ncols + ncols elements)
bem_status general_gram_apply(bem_ctx* h, int mode, const cplx* in, cplx* out, cplx* tmp, size_t tmp_elems, int64_t N,
                              int64_t ncols, int64_t si, int64_t sc, bool conj_out);
size_t cyc_factor_bytes(int64_t N);
// h->Q, h->GQ, h->gm of a general mesh (nc columns, with the constant mode when inc)
bem_status general_filter_basis(bem_ctx* h, int64_t nc, int inc);
void general_basis_plan(int64_t N, int64_t n, double perimeter, int64_t* p_out, int* iters_out, double* sigma_out,
                        double* bound_out);
bem_status launch_copy2d(bem_ctx* h, void* dst, int64_t ldd, const void* src, int64_t lds,
                         int64_t rows, int64_t cols, size_t elem);
