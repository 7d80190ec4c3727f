// Mixed-precision path (placeholder until the tcgen05 kernels land).
#include "tc_gemm.h"

bem_status tc_prepare_operators(bem_ctx* h) { return bem_fail(h, BEM_E_UNSUPPORTED, "mixed path not built"); }
bem_status tc_product_left(bem_ctx* h, int, const double*, const cplx*, int64_t, cplx*) {
    return bem_fail(h, BEM_E_UNSUPPORTED, "mixed path not built");
}
bem_status tc_product_right(bem_ctx* h, int, const cplx*, int64_t, int64_t, cplx*, int64_t) {
    return bem_fail(h, BEM_E_UNSUPPORTED, "mixed path not built");
}
bem_status tc_prepare_solve(bem_ctx* h) { return bem_fail(h, BEM_E_UNSUPPORTED, "mixed path not built"); }
bem_status tc_solve_refined(bem_ctx* h, const cplx*, int64_t, cplx*, int64_t, int64_t, int32_t*, double*) {
    return bem_fail(h, BEM_E_UNSUPPORTED, "mixed path not built");
}
void tc_release_operands(bem_ctx*) {}
void tc_release_solve(bem_ctx*) {}
void tc_destroy(bem_ctx*) {}
