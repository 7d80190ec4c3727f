// Mixed-precision (split-bf16, tcgen05) products of the solver (internal interface).
#pragma once

#include "common.cuh"

enum { TC_OP_S = 0, TC_OP_W = 1, TC_OP_D = 2 };

// Slices the assembled operators for the tensor-core products (after bem_assemble).
bem_status tc_prepare_operators(bem_ctx* h);
// out (nc x N, ld nc) = L * OP, with L = Q^T (Qreal: N x nc real) or L = Y (nc x N complex).
bem_status tc_product_left(bem_ctx* h, int op, const double* Qreal, const cplx* Y, int64_t nc, cplx* out);
// out (N x nrhs, ld) = OP * y (y: N x nrhs, ld N).
bem_status tc_product_right(bem_ctx* h, int op, const cplx* y, int64_t ldy, int64_t nrhs, cplx* out, int64_t ld);
// Slices U and V^H for the Woodbury products (after factor).
bem_status tc_prepare_solve(bem_ctx* h);
// U = Qs E_r and V^H = E_r^H Bs (compression factors) as split-bf16 products.
bem_status tc_compress_factors(bem_ctx* h, const double* Qs, cplx* U, cplx* Vh);
// Kt = beta^-1 V^H U (r x r, ld r) as a split-bf16 product (after tc_prepare_solve).
bem_status tc_core_product(bem_ctx* h, cplx* Kt);
// Woodbury solve with split-bf16 products and FP64 residual refinement.
bem_status tc_solve_refined(bem_ctx* h, const cplx* v, int64_t ldv, cplx* x, int64_t ldx, int64_t nrhs,
                            int32_t* iters, double* max_rel_resid);
void tc_release_operands(bem_ctx* h);
void tc_release_solve(bem_ctx* h);
void tc_destroy(bem_ctx* h);
