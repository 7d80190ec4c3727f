// C ABI entry points (include/bem.h): the stage machine of the filtered Calderon fast
// direct solver, Sec. IV of Henry et al. (EuCAP 2023), on top of the kernels in
// assemble.cu, linalg.cu and tc_gemm.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "tc_gemm.h"

bem_status bem_fail(bem_ctx* h, bem_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

bem_status bem_cuda_check(bem_ctx* h, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return bem_fail(h, BEM_E_NOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return bem_fail(h, BEM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t bem_dmalloc(bem_ctx* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (!h->dev_alloc) return cudaMalloc(p, bytes);
    *p = h->dev_alloc(bytes, h->alloc_ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void bem_dfree(bem_ctx* h, void* p) {
    if (!p) return;
    if (h->dev_free) h->dev_free(p, h->alloc_ctx);
    else cudaFree(p);
}

cudaError_t bem_dmalloc_async(bem_ctx* h, void** p, size_t bytes) {
    if (!h->dev_alloc) {
        *p = nullptr;
        return cudaMallocAsync(p, bytes ? bytes : 256, h->stream);
    }
    return bem_dmalloc(h, p, bytes);
}

void bem_dfree_async(bem_ctx* h, void* p) {
    if (!p) return;
    if (h->dev_free) h->dev_free(p, h->alloc_ctx);
    else cudaFreeAsync(p, h->stream);
}

bem_status bem_workspace(bem_ctx* h, size_t bytes, void** out) {
    void** w = h->rhs_aux ? &h->work2 : &h->work;
    size_t* wb = h->rhs_aux ? &h->work2_bytes : &h->work_bytes;
    if (bytes > *wb) {
        if (*w) {
            cudaStreamSynchronize(h->stream);          // the stream that uses this workspace
            bem_dfree(h, *w);
            *w = nullptr;
            *wb = 0;
        }
        size_t want = std::max(bytes, (size_t)1 << 20);
        BEM_CUDA(h, bem_dmalloc(h, w, want));
        *wb = want;
    }
    *out = *w;
    return BEM_OK;
}

// carve sub-buffers (256-byte aligned) out of one workspace request
struct Carve {
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

static void free_ptr(bem_ctx* h, void** p) {
    if (*p) { bem_dfree(h, *p); *p = nullptr; }
    h->caps.erase(p);
}

// stage buffers keep their allocation from step to step (cudaFree would wait for the whole
// device, other streams included); a buffer is reallocated only when it has to grow
static bem_status ensure_alloc(bem_ctx* h, void** p, size_t bytes) {
    auto it = h->caps.find(p);
    if (*p && it != h->caps.end() && it->second >= bytes) return BEM_OK;
    if (*p) {
        BEM_CUDA(h, cudaStreamSynchronize(h->stream));
        free_ptr(h, p);
    }
    BEM_CUDA(h, bem_dmalloc(h, p, bytes));
    h->caps[p] = bytes;
    return BEM_OK;
}

static bem_status check_dev_err(bem_ctx* h) {
    int e = 0;
    BEM_CUDA(h, cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (e) {
        BEM_CUDA(h, cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
        if (e & DEVERR_TIMEOUT) return bem_fail(h, BEM_E_TIMEOUT, "a device-side wait timed out");
        if (e & DEVERR_SINGULAR) return bem_fail(h, BEM_E_SINGULAR, "zero pivot in the Woodbury core");
        return bem_fail(h, BEM_E_CUDA, "device error flag set");
    }
    return BEM_OK;
}

cudaEvent_t bem_event_get(bem_ctx* h) {
    if (!h->evpool.empty()) {
        cudaEvent_t e = h->evpool.back();
        h->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static std::mutex g_tab_mutex;
static bool g_tab_done[64] = {false};

extern "C" {

void bem_default_options(bem_options* opt) {
    if (!opt) return;
    opt->prec = BEM_FP64;
    opt->include_kernel_mode = 1;
    opt->refine_rtol = 1e-10;
    opt->max_refine = 6;
    opt->split_slices = 0;
    opt->rhs_slices = 0;
    opt->solve_slices = 0;
    opt->filter_tile_n = 0;
    opt->filter_split_k = 0;
    opt->rhs_tile_n = 0;
    opt->rhs_split_k = 0;
    opt->asm_tile = 0;
}

bem_status bem_create(bem_handle* out, int device, void* cuda_stream, const bem_options* opt,
                      bem_dev_alloc_fn dev_alloc, bem_dev_free_fn dev_free, void* alloc_ctx) {
    if (!out) return BEM_E_INVALID;
    *out = nullptr;
    if ((dev_alloc == nullptr) != (dev_free == nullptr)) return BEM_E_INVALID;
    bem_ctx* h = new (std::nothrow) bem_ctx();
    if (!h) return BEM_E_NOMEM;
    h->dev_alloc = dev_alloc;
    h->dev_free = dev_free;
    h->alloc_ctx = alloc_ctx;
    if (opt) h->opt = *opt; else bem_default_options(&h->opt);
    if (h->opt.prec != BEM_FP64 && h->opt.prec != BEM_MIXED_BF16) { delete h; return BEM_E_INVALID; }
    if (h->opt.refine_rtol <= 0.0) h->opt.refine_rtol = 1e-10;
    if (h->opt.max_refine < 0) h->opt.max_refine = 0;
    if (h->opt.asm_tile != 0 && h->opt.asm_tile != 15 && h->opt.asm_tile != 23 && h->opt.asm_tile != 31) {
        delete h;
        return BEM_E_INVALID;
    }
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete h; return BEM_E_CUDA; }
    {
        std::lock_guard<std::mutex> lk(g_tab_mutex);
        if (device < 0 || device >= 64) { delete h; return BEM_E_INVALID; }
        if (!g_tab_done[device]) {
            if (init_gauss_tables() != cudaSuccess) { delete h; return BEM_E_CUDA; }
            g_tab_done[device] = true;
        }
    }
    if (bem_dmalloc(h, (void**)&h->dev_err, sizeof(int)) != cudaSuccess ||
        bem_dmalloc(h, (void**)&h->bar, 4 * sizeof(unsigned)) != cudaSuccess ||
        bem_dmalloc(h, (void**)&h->qpts, sizeof(unsigned long long)) != cudaSuccess) {
        bem_dfree(h, h->dev_err);
        bem_dfree(h, h->bar);
        bem_dfree(h, h->qpts);
        delete h;
        return BEM_E_NOMEM;
    }
    cudaMemset(h->dev_err, 0, sizeof(int));
    cudaMemset(h->bar, 0, 4 * sizeof(unsigned));
    cudaMemset(h->qpts, 0, sizeof(unsigned long long));
    *out = h;
    return BEM_OK;
}

// Releases the buffers of the stages from from_stage on.  Recomputing a stage on a problem
// of the same size keeps them (the stage counter says what they hold; ensure_alloc reuses or
// grows them), so a step frees nothing; a new N (from_stage <= 1) or bem_destroy frees all.
static void free_stage_buffers(bem_ctx* h, int from_stage) {
    if (from_stage > 1) return;
    free_ptr(h, (void**)&h->S); free_ptr(h, (void**)&h->W); free_ptr(h, (void**)&h->D);
    free_ptr(h, (void**)&h->rexp); h->rexp_valid = false;
    free_ptr(h, (void**)&h->k1); free_ptr(h, (void**)&h->kpart); h->kpart_slots = 0; h->k1_valid = false;
    free_ptr(h, (void**)&h->seg);
    free_ptr(h, (void**)&h->gfac);
    h->general = false;
    tc_release_operands(h);
    free_ptr(h, (void**)&h->B); free_ptr(h, (void**)&h->gm); free_ptr(h, (void**)&h->Q);
    free_ptr(h, (void**)&h->GQ);
    free_ptr(h, (void**)&h->Bs);
    free_ptr(h, (void**)&h->sigma); free_ptr(h, (void**)&h->E);
    free_ptr(h, (void**)&h->U); free_ptr(h, (void**)&h->Vh);
    free_ptr(h, (void**)&h->K); free_ptr(h, (void**)&h->piv);
    tc_release_solve(h);
}

bem_status bem_destroy(bem_handle h) {
    if (!h) return BEM_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->hi) cudaStreamSynchronize(h->hi);
    free_stage_buffers(h, 0);
    tc_destroy(h);
    free_ptr(h, &h->work);
    free_ptr(h, &h->work2);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->hi) cudaStreamDestroy(h->hi);
    free_ptr(h, (void**)&h->btab);
    free_ptr(h, (void**)&h->btabf);
    free_ptr(h, (void**)&h->dev_err);
    free_ptr(h, (void**)&h->bar);
    free_ptr(h, (void**)&h->qpts);
    delete h;
    return BEM_OK;
}

const char* bem_last_error(bem_handle h) { return h ? h->err.c_str() : "null handle"; }

bem_status bem_set_stream(bem_handle h, void* s) {
    if (!h) return BEM_E_INVALID;
    h->stream = (cudaStream_t)s;
    return BEM_OK;
}

// everything of bem_assemble before the tiles: checks, buffers, geometry (one stream sync for
// the mesh check)
static bem_status assemble_begin(bem_handle h, const double* verts, int64_t N, double k, unsigned ops) {
    if (!verts || N < 16 || N > (1 << 20) || !(k > 0.0) || !std::isfinite(k) || (ops & ~7u) || !(ops & 3u))
        return bem_fail(h, BEM_E_INVALID, "bem_assemble: need verts, 16 <= N <= 2^20, k > 0, ops with S or W");
    BEM_CUDA(h, cudaSetDevice(h->device));
    if (N != h->N) free_stage_buffers(h, 0);
    else free_stage_buffers(h, 2);
    h->stage = 0;
    const size_t NN = (size_t)N * (size_t)N;
    bem_status st;
    if ((st = ensure_alloc(h, (void**)&h->seg, sizeof(double) * 5 * N)) != BEM_OK) return st;
    // S and W are always assembled together (the EFIE needs both); D on request
    if ((st = ensure_alloc(h, (void**)&h->S, sizeof(cplx) * NN)) != BEM_OK) return st;
    if ((st = ensure_alloc(h, (void**)&h->W, sizeof(cplx) * NN)) != BEM_OK) return st;
    if (ops & BEM_OP_D) {
        if ((st = ensure_alloc(h, (void**)&h->D, sizeof(cplx) * NN)) != BEM_OK) return st;
    } else {
        free_ptr(h, (void**)&h->D);
    }
    h->N = N;
    h->k = k;
    double* stats = nullptr;
    Carve cv; cv.add((void**)&stats, 3 * sizeof(double));
    if ((st = cv.commit(h)) != BEM_OK) return st;
    if ((st = launch_geometry(h, verts, N, stats)) != BEM_OK) return st;
    double hs[3];
    BEM_CUDA(h, cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, h->stream));
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    const double hmean = hs[2] / (double)N;
    if (!(hs[0] > 0.0) || !std::isfinite(hs[2]))
        return bem_fail(h, BEM_E_INVALID, "bem_assemble: degenerate or non-finite vertices");
    if (k * hs[1] > 2.0)
        return bem_fail(h, BEM_E_UNSUPPORTED, "bem_assemble: k h > 2 (mesh too coarse for this frequency)");
    h->hbar = hmean;
    h->hmax = hs[1];
    // chords equal to rounding (1e-10 of the mean): circulant G and L, Fourier filter basis;
    // otherwise the general cyclic tridiagonal G and L of mesh.cu
    h->general = (hs[1] - hs[0]) > 1e-10 * hmean;
    if (h->general) {
        if ((st = ensure_alloc(h, (void**)&h->gfac, cyc_factor_bytes(N))) != BEM_OK) return st;
        if ((st = launch_cyc_factor(h, 0.0, 1.0, h->gfac)) != BEM_OK) return st;
    } else {
        free_ptr(h, (void**)&h->gfac);
    }
    h->ops = BEM_OP_S | BEM_OP_W | (ops & BEM_OP_D);
    return BEM_OK;
}

// after the tiles: the mixed path's digit slices
static bem_status assemble_end(bem_handle h) {
    if (h->opt.prec == BEM_MIXED_BF16) {
        bem_status st = tc_prepare_operators(h);
        if (st != BEM_OK) return st;
    }
    h->stage = 1;
    return BEM_OK;
}

bem_status bem_assemble(bem_handle h, const double* verts, int64_t N, double k, unsigned ops) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    bem_status st;
    if ((st = assemble_begin(h, verts, N, k, ops)) != BEM_OK) return st;
    if ((st = launch_assemble(h, h->ops)) != BEM_OK) return st;
    return assemble_end(h);
}

bem_status bem_assemble_batch(bem_handle* hs, int64_t nprob, const double* const* verts, const int64_t* Ns,
                              const double* ks) {
    if (!hs || !verts || !Ns || !ks || nprob < 1 || nprob > 65536) return BEM_E_INVALID;
    for (int64_t q = 0; q < nprob; ++q) {
        if (!hs[q]) return BEM_E_INVALID;
        if (hs[q]->device != hs[0]->device)
            return bem_fail(hs[q], BEM_E_INVALID, "bem_assemble_batch: every handle must be on the same device");
        for (int64_t r = 0; r < q; ++r)
            if (hs[r] == hs[q]) return bem_fail(hs[q], BEM_E_INVALID, "bem_assemble_batch: a handle appears twice");
    }
    for (int64_t q = 0; q < nprob; ++q) {
        hs[q]->err.clear();
        bem_status st = assemble_begin(hs[q], verts[q], Ns[q], ks[q], BEM_OP_S | BEM_OP_W);
        if (st != BEM_OK) {
            if (q > 0) bem_fail(hs[0], st, "bem_assemble_batch: problem " + std::to_string(q) + ": " + hs[q]->err);
            return st;
        }
    }
    BEM_CUDA(hs[0], cudaSetDevice(hs[0]->device));
    bem_status st = launch_assemble_batch(hs, (int)nprob);
    if (st != BEM_OK) return st;
    for (int64_t q = 0; q < nprob; ++q)
        if ((st = assemble_end(hs[q])) != BEM_OK) return st;
    return BEM_OK;
}

bem_status filter_apply(bem_handle h, int64_t n_modes, double alpha) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "filter_apply: call bem_assemble first");
    const int64_t N = h->N;
    if (n_modes < 3 || (n_modes % 2) == 0 || n_modes > N - 1 || n_modes > 1023)
        return bem_fail(h, BEM_E_INVALID, "filter_apply: n_modes must be odd, 3 <= n <= min(N-1, 1023)");
    if (!std::isfinite(alpha) || alpha < 0.0)
        return bem_fail(h, BEM_E_INVALID, "filter_apply: alpha must be finite and >= 0");
    if (alpha != 0.0 && !h->D)
        return bem_fail(h, BEM_E_INVALID, "filter_apply: alpha != 0 needs D (assemble with BEM_OP_D)");
    BEM_CUDA(h, cudaSetDevice(h->device));
    free_stage_buffers(h, 2);
    h->stage = 1;
    const int inc = h->opt.include_kernel_mode ? 1 : 0;
    const int64_t nc = inc ? n_modes : n_modes - 1;
    bem_status st;
    if ((st = ensure_alloc(h, (void**)&h->B, sizeof(cplx) * nc * N)) != BEM_OK) return st;
    if ((st = ensure_alloc(h, (void**)&h->gm, sizeof(double) * nc)) != BEM_OK) return st;
    if ((st = ensure_alloc(h, (void**)&h->Q, sizeof(double) * nc * N)) != BEM_OK) return st;
    h->n = n_modes;
    h->ncols = nc;
    h->M = (n_modes - 1) / 2;
    h->alpha = alpha;
    h->beta = (1.0 + 2.0 * alpha) / 4.0;
    if (h->general) {
        // the lowest eigenvectors of the pencil (L, G), G-orthonormal (gm = 1), and G Q
        if ((st = ensure_alloc(h, (void**)&h->GQ, sizeof(double) * nc * N)) != BEM_OK) return st;
        if ((st = general_filter_basis(h, nc, inc)) != BEM_OK) return st;
    } else {
        if ((st = launch_fourier_basis(h, h->Q, N, nc, inc, h->gm, h->hbar)) != BEM_OK) return st;
    }
    cplx *Y1 = nullptr, *tmp = nullptr, *cfix = nullptr;
    Carve cv;
    cv.add((void**)&Y1, sizeof(cplx) * nc * N);
    cv.add((void**)&tmp, sizeof(cplx) * nc * N);
    cv.add((void**)&cfix, sizeof(cplx) * (N + nc));
    if ((st = cv.commit(h)) != BEM_OK) return st;
    if (h->opt.prec == BEM_MIXED_BF16) {
        // Y1 = Q^T S and B = Y2 N as split-bf16 tensor-core products
        if ((st = tc_product_left(h, TC_OP_S, h->Q, nullptr, nc, Y1)) != BEM_OK) return st;
    } else {
        // Y1 = Q^T S  (ncols x N)
        h->tag = "gemm_filter_QtS";
        if ((st = dzgemm_realA(h, OP_T, nc, N, N, 1.0, h->Q, N, h->S, N, 0.0, Y1, nc)) != BEM_OK) return st;
    }
    // Y2 = Y1 G^-1 (along the N index of each row)
    if ((st = apply_gram_inverse(h, 0, Y1, Y1, tmp, N, nc, nc, 1, h->hbar, false)) != BEM_OK) return st;
    if (h->opt.prec == BEM_MIXED_BF16) {
        if ((st = tc_product_left(h, TC_OP_W, nullptr, Y1, nc, h->B)) != BEM_OK) return st;
        // the product's action on the constant vector, from N's row sums
        if ((st = launch_const_correction(h, h->W, h->k1_valid ? h->k1 : nullptr, Y1, h->B, nc, N, cfix)) != BEM_OK)
            return st;
        if (alpha != 0.0) {
            if ((st = tc_product_left(h, TC_OP_D, h->Q, nullptr, nc, tmp)) != BEM_OK) return st;
            if ((st = launch_axpby(h, h->B, nc, tmp, nc, cmk(-alpha, 0), cmk(1, 0), nc, N)) != BEM_OK) return st;
        }
    } else {
        // B = Y2 N  (- alpha Q^T D)
        h->tag = "gemm_filter_YN";
        if ((st = zgemm(h, OP_N, OP_N, nc, N, N, cmk(1, 0), Y1, nc, h->W, N, cmk(0, 0), h->B, nc)) != BEM_OK) return st;
        // the product's action on the constant vector from N's exact row sums (the stored
        // entries' rounding moves them by up to 2^-53 sum_j |N_ij|, O(k^-2) of them at low k)
        if (h->k1_valid)
            if ((st = launch_const_correction(h, h->W, h->k1, Y1, h->B, nc, N, cfix)) != BEM_OK) return st;
        h->tag = "gemm_filter_QtD";
        if (alpha != 0.0)
            if ((st = dzgemm_realA(h, OP_T, nc, N, N, -alpha, h->Q, N, h->D, N, 1.0, h->B, nc)) != BEM_OK) return st;
    }
    // B = diag(1/g) B - Q^T/4  (general mesh: B - (G Q)^T/4, g = 1)
    if ((st = launch_finish_B(h, h->B, h->gm, h->general ? h->GQ : h->Q, nc, N)) != BEM_OK) return st;
    h->stage = 2;
    return BEM_OK;
}

}  // extern "C"

// compress_compact's work; after_qr runs once the pivoted QR is enqueued (the fork point of
// bem_factor_rhs_planewave: nothing after it reads what the right-hand sides write)
template <class AfterQR>
static bem_status compress_impl(bem_ctx* h, double rel_tol, int64_t* rank_out, AfterQR after_qr) {
    if (h->stage < 2) return bem_fail(h, BEM_E_INVALID, "compress_compact: call filter_apply first");
    if (!std::isfinite(rel_tol) || rel_tol >= 1.0)
        return bem_fail(h, BEM_E_INVALID, "compress_compact: rel_tol must be < 1");
    BEM_CUDA(h, cudaSetDevice(h->device));
    free_stage_buffers(h, 3);
    h->stage = 2;
    const int64_t N = h->N, nc = h->ncols;
    bem_status st;
    if ((st = ensure_alloc(h, (void**)&h->sigma, sizeof(double) * nc)) != BEM_OK) return st;
    if ((st = ensure_alloc(h, (void**)&h->E, sizeof(cplx) * nc * nc)) != BEM_OK) return st;
    if ((st = ensure_alloc(h, (void**)&h->Bs, sizeof(cplx) * nc * N)) != BEM_OK) return st;
    cplx *X = nullptr, *R = nullptr;
    double* Qs = nullptr;
    int* perm = nullptr;
    void* jac = nullptr;
    Carve cv;
    cv.add((void**)&X, sizeof(cplx) * nc * N);
    cv.add((void**)&R, sizeof(cplx) * nc * nc);
    cv.add((void**)&Qs, sizeof(double) * nc * N);
    cv.add((void**)&perm, sizeof(int) * nc);
    cv.add(&jac, jacobi_scratch_bytes((int)nc));
    cplx* gtmp = nullptr;                      // scratch of the general mesh's chunked Gram solve
    if (h->general) cv.add((void**)&gtmp, sizeof(cplx) * nc * N);
    if ((st = cv.commit(h)) != BEM_OK) return st;
    // Bs = diag(sqrt g) B ;  X = (Bs F^-1)^H  (N x nc, stored with row stride nc)
    if ((st = launch_row_scale(h, h->B, h->Bs, h->gm, 1, nc, N, nc)) != BEM_OK) return st;
    if ((st = apply_gram_inverse(h, 1, h->Bs, X, gtmp, N, nc, nc, 1, h->hbar, true)) != BEM_OK) return st;
    // B^ = X^H: pivoted QR X P = Q R, then the left singular vectors of R^H, rows permuted
    // back by P, are those of B^
    if ((st = launch_house_qr(h, X, N, (int)nc, R, perm, h->opt.prec == BEM_MIXED_BF16)) != BEM_OK) return st;
    if ((st = after_qr()) != BEM_OK) return st;
    if ((st = launch_jacobi_svd(h, R, (int)nc, perm, h->sigma, h->E, jac)) != BEM_OK) return st;
    std::vector<double> sig(nc);
    BEM_CUDA(h, cudaMemcpyAsync(sig.data(), h->sigma, sizeof(double) * nc, cudaMemcpyDeviceToHost, h->stream));
    if ((st = check_dev_err(h)) != BEM_OK) return st;
    h->sigma_max = sig[0];
    int64_t r = 0;
    for (int64_t i = 0; i < nc; ++i) {
        if (rel_tol > 0.0 ? (sig[i] >= rel_tol * sig[0]) : (sig[i] > 0.0)) ++r;
    }
    if (r < 1) r = 1;
    h->r = r;
    if ((st = ensure_alloc(h, (void**)&h->U, sizeof(cplx) * N * r)) != BEM_OK) return st;
    if ((st = ensure_alloc(h, (void**)&h->Vh, sizeof(cplx) * r * N)) != BEM_OK) return st;
    // U = Q diag(g^-1/2) E_r ;  V^H = E_r^H diag(g^1/2) B
    if ((st = launch_scale_real_cols(h, h->Q, Qs, h->gm, -1, N, nc)) != BEM_OK) return st;
    if (h->opt.prec == BEM_MIXED_BF16) {
        if ((st = tc_compress_factors(h, Qs, h->U, h->Vh)) != BEM_OK) return st;
    } else {
        h->tag = "gemm_compress_UVh";
        if ((st = dzgemm_realA(h, OP_N, N, r, nc, 1.0, Qs, N, h->E, nc, 0.0, h->U, N)) != BEM_OK) return st;
        if ((st = zgemm(h, OP_C, OP_N, r, N, nc, cmk(1, 0), h->E, nc, h->Bs, nc, cmk(0, 0), h->Vh, r)) != BEM_OK)
            return st;
    }
    if (rank_out) *rank_out = r;
    h->stage = 3;
    return BEM_OK;
}

extern "C" {

bem_status compress_compact(bem_handle h, double rel_tol, int64_t* rank_out) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    return compress_impl(h, rel_tol, rank_out, [] { return BEM_OK; });
}

bem_status factor(bem_handle h) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 3) return bem_fail(h, BEM_E_INVALID, "factor: call compress_compact first");
    BEM_CUDA(h, cudaSetDevice(h->device));
    free_stage_buffers(h, 4);
    h->stage = 3;
    const int64_t N = h->N, r = h->r;
    bem_status st;
    if ((st = ensure_alloc(h, (void**)&h->K, sizeof(cplx) * r * r)) != BEM_OK) return st;
    cplx* Kt = nullptr;
    void* gj = nullptr;
    Carve cv;
    cv.add((void**)&Kt, sizeof(cplx) * r * r);
    cv.add(&gj, gauss_jordan_scratch_bytes((int)r));
    if ((st = cv.commit(h)) != BEM_OK) return st;
    // K = I_r + beta^-1 V^H U, stored as its inverse
    if (h->opt.prec == BEM_MIXED_BF16) {
        // slices of U and V^H serve the core product here and every later solve
        if ((st = tc_prepare_solve(h)) != BEM_OK) return st;
        if ((st = tc_core_product(h, Kt)) != BEM_OK) return st;
    } else {
        h->tag = "gemm_factor_VhU";
        if ((st = zgemm(h, OP_N, OP_N, r, r, N, cmk(1.0 / h->beta, 0), h->Vh, r, h->U, N, cmk(0, 0), Kt, r)) != BEM_OK)
            return st;
    }
    if ((st = launch_add_identity(h, Kt, r, (int)r, cmk(1, 0))) != BEM_OK) return st;
    if ((st = launch_gauss_jordan(h, Kt, h->K, (int)r, gj)) != BEM_OK) return st;
    if ((st = check_dev_err(h)) != BEM_OK) return st;
    h->stage = 4;
    return BEM_OK;
}

}  // extern "C"

// f (and hz for the CFIE) by `make`, then v = G^-1 S G^-1 f - alpha G^-1 hz
template <class Make>
static bem_status rhs_common(bem_ctx* h, const char* who, int64_t nrhs, void* f_out, void* v_out, int64_t ld,
                             Make make) {
    const int64_t N = h->N;
    bem_status st;
    // every internal block uses the caller's leading dimension ld
    cplx *f = (cplx*)f_out, *hz = nullptr, *y = nullptr, *tmp = nullptr;
    Carve cv;
    if (!f) cv.add((void**)&f, sizeof(cplx) * ld * nrhs);
    if (v_out) {
        if (h->alpha != 0.0) cv.add((void**)&hz, sizeof(cplx) * ld * nrhs);
        cv.add((void**)&y, sizeof(cplx) * ld * nrhs);
        cv.add((void**)&tmp, sizeof(cplx) * ld * nrhs);
    }
    if ((st = cv.commit(h)) != BEM_OK) return st;
    if ((st = make(f, hz)) != BEM_OK) return st;
    if (!v_out) return BEM_OK;
    cplx* v = (cplx*)v_out;
    // y = G^-1 f
    if ((st = apply_gram_inverse(h, 0, f, y, tmp, N, nrhs, 1, ld, h->hbar, false)) != BEM_OK) return st;
    // v <- S y (- alpha h2), then v <- G^-1 v
    if (h->opt.prec == BEM_MIXED_BF16) {
        if ((st = tc_product_right(h, TC_OP_S, y, ld, nrhs, v, ld)) != BEM_OK) return st;
    } else {
        h->tag = "gemm_rhs_SY";
        if ((st = zgemm(h, OP_N, OP_N, N, nrhs, N, cmk(1, 0), h->S, N, y, ld, cmk(0, 0), v, ld)) != BEM_OK) return st;
    }
    if (hz) {
        if ((st = launch_axpby(h, v, ld, hz, ld, cmk(-h->alpha, 0), cmk(1, 0), N, nrhs)) != BEM_OK) return st;
    }
    (void)who;
    return apply_gram_inverse(h, 0, v, v, tmp, N, nrhs, 1, ld, h->hbar, false);
}

extern "C" {

bem_status bem_rhs_planewave(bem_handle h, const double* angles, int64_t nrhs, void* f_out, void* v_out, int64_t ld) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_rhs_planewave: call bem_assemble first");
    if (!angles || nrhs < 1 || nrhs > 65535 || ld < h->N)
        return bem_fail(h, BEM_E_INVALID, "bem_rhs_planewave: need angles, 1 <= nrhs <= 65535, ld >= N");
    if (!f_out && !v_out) return BEM_OK;
    BEM_CUDA(h, cudaSetDevice(h->device));
    return rhs_common(h, "bem_rhs_planewave", nrhs, f_out, v_out, ld,
                      [&](cplx* f, cplx* hz) { return launch_rhs(h, angles, nrhs, f, hz, ld); });
}

bem_status bem_rhs_pointsource(bem_handle h, const double* src_xy, int64_t nsrc, void* f_out, void* v_out,
                               int64_t ld) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_rhs_pointsource: call bem_assemble first");
    if (!src_xy || nsrc < 1 || nsrc > 65535 || ld < h->N)
        return bem_fail(h, BEM_E_INVALID, "bem_rhs_pointsource: need sources, 1 <= nsrc <= 65535, ld >= N");
    if (!f_out && !v_out) return BEM_OK;
    BEM_CUDA(h, cudaSetDevice(h->device));
    return rhs_common(h, "bem_rhs_pointsource", nsrc, f_out, v_out, ld,
                      [&](cplx* f, cplx* hz) { return launch_rhs_point(h, src_xy, nsrc, f, hz, ld); });
}

// compress_compact, factor and bem_rhs_planewave in one call, with the right-hand sides on a
// second stream of the handle: forked once the pivoted QR is enqueued, they run beside the
// Jacobi SVD, the compression products and the Gauss-Jordan factor (kernels small enough to
// share SMs with the split product's CTAs), and are joined to the handle's stream before
// the call returns.  Their scratch (workspace, the product's B operand) is their own.
bem_status bem_factor_rhs_planewave(bem_handle h, double rel_tol, const double* angles, int64_t nrhs, void* f_out,
                                    void* v_out, int64_t ld, int64_t* rank_out) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 2) return bem_fail(h, BEM_E_INVALID, "bem_factor_rhs_planewave: call filter_apply first");
    if (!angles || !v_out || nrhs < 1 || nrhs > 65535 || ld < h->N)
        return bem_fail(h, BEM_E_INVALID, "bem_factor_rhs_planewave: need angles, v, 1 <= nrhs <= 65535, ld >= N");
    BEM_CUDA(h, cudaSetDevice(h->device));
    if (!h->aux) BEM_CUDA(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    if (!h->hi) {
        int least = 0, greatest = 0;
        BEM_CUDA(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BEM_CUDA(h, cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, greatest));
    }
    cudaStream_t mainst = h->stream;
    cudaEvent_t done = nullptr;
    bool forked = false;
    bem_status rst = BEM_OK;
    std::string rerr;
    auto fork_rhs = [&]() -> bem_status {
        cudaEvent_t qr = bem_event_get(h);
        BEM_CUDA(h, cudaEventRecord(qr, mainst));
        BEM_CUDA(h, cudaStreamWaitEvent(h->aux, qr, 0));
        BEM_CUDA(h, cudaStreamWaitEvent(h->hi, qr, 0));
        h->evpool.push_back(qr);            // the waits took the record; the event may be reused
        forked = true;
        h->stream = h->aux;
        h->rhs_aux = true;
        rst = rhs_common(h, "bem_factor_rhs_planewave", nrhs, f_out, v_out, ld,
                         [&](cplx* f, cplx* hz) { return launch_rhs(h, angles, nrhs, f, hz, ld); });
        if (rst != BEM_OK) rerr = h->err;
        done = bem_event_get(h);
        cudaEventRecord(done, h->aux);
        h->stream = h->hi;                  // the rest of the compression, and the factor
        h->rhs_aux = false;
        return BEM_OK;                      // the right-hand sides' status is reported after the join
    };
    bem_status st = compress_impl(h, rel_tol, rank_out, fork_rhs);
    h->rhs_aux = false;
    if (st == BEM_OK) st = factor(h);
    h->stream = mainst;
    if (forked) {
        cudaEvent_t hd = bem_event_get(h);
        cudaEventRecord(hd, h->hi);
        cudaStreamWaitEvent(mainst, hd, 0);
        h->evpool.push_back(hd);
    }
    if (done) {
        cudaStreamWaitEvent(mainst, done, 0);
        h->evpool.push_back(done);
    }
    if (st == BEM_OK && rst != BEM_OK) {
        h->err = rerr;
        st = rst;
    }
    return st;
}

// x = v/beta - beta^-2 U Kinv V^H v, all FP64 products
static bem_status woodbury_fp64(bem_ctx* h, const cplx* v, int64_t ldv, cplx* x, int64_t ldx, int64_t nrhs,
                                cplx* T, cplx* T2) {
    const int64_t N = h->N, r = h->r;
    bem_status st;
    h->tag = "gemm_solve";
    if ((st = zgemm(h, OP_N, OP_N, r, nrhs, N, cmk(1, 0), h->Vh, r, v, ldv, cmk(0, 0), T, r)) != BEM_OK) return st;
    if ((st = zgemm(h, OP_N, OP_N, r, nrhs, r, cmk(1, 0), h->K, r, T, r, cmk(0, 0), T2, r)) != BEM_OK) return st;
    if ((st = launch_axpby(h, x, ldx, v, ldv, cmk(1.0 / h->beta, 0), cmk(0, 0), N, nrhs)) != BEM_OK) return st;
    return zgemm(h, OP_N, OP_N, N, nrhs, r, cmk(-1.0 / (h->beta * h->beta), 0), h->U, N, T2, r, cmk(1, 0), x, ldx);
}

// rho = v - (beta x + U V^H x), FP64
static bem_status residual_fp64(bem_ctx* h, const cplx* v, int64_t ldv, const cplx* x, int64_t ldx, int64_t nrhs,
                                cplx* rho, cplx* T) {
    const int64_t N = h->N, r = h->r;
    bem_status st;
    h->tag = "gemm_residual";
    if ((st = zgemm(h, OP_N, OP_N, r, nrhs, N, cmk(1, 0), h->Vh, r, x, ldx, cmk(0, 0), T, r)) != BEM_OK) return st;
    if ((st = launch_copy2d(h, rho, N, v, ldv, N, nrhs, sizeof(cplx))) != BEM_OK) return st;
    if ((st = launch_axpby(h, rho, N, x, ldx, cmk(-h->beta, 0), cmk(1, 0), N, nrhs)) != BEM_OK) return st;
    return zgemm(h, OP_N, OP_N, N, nrhs, r, cmk(-1, 0), h->U, N, T, r, cmk(1, 0), rho, N);
}

bem_status solve_many(bem_handle h, const void* v_dev, int64_t ldv, void* x_dev, int64_t ldx, int64_t nrhs,
                      int32_t* iters_out, double* max_rel_resid_out) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 4) return bem_fail(h, BEM_E_INVALID, "solve_many: call factor first");
    const int64_t N = h->N, r = h->r;
    if (!v_dev || !x_dev || nrhs < 1 || nrhs > (1 << 24) || ldv < N || ldx < N || v_dev == x_dev)
        return bem_fail(h, BEM_E_INVALID, "solve_many: need v, x (not aliased), nrhs >= 1, ld >= N");
    BEM_CUDA(h, cudaSetDevice(h->device));
    const cplx* v = (const cplx*)v_dev;
    cplx* x = (cplx*)x_dev;
    bem_status st;
    if (h->opt.prec == BEM_MIXED_BF16) {
        int32_t it = 0;
        double res = 0.0;
        st = tc_solve_refined(h, v, ldv, x, ldx, nrhs, &it, &res);
        if (iters_out) *iters_out = it;
        if (max_rel_resid_out) *max_rel_resid_out = res;
        return st;
    }
    cplx *T = nullptr, *T2 = nullptr, *rho = nullptr;
    Carve cv;
    cv.add((void**)&T, sizeof(cplx) * r * nrhs);
    cv.add((void**)&T2, sizeof(cplx) * r * nrhs);
    if (max_rel_resid_out) cv.add((void**)&rho, sizeof(cplx) * N * nrhs);
    if ((st = cv.commit(h)) != BEM_OK) return st;
    if ((st = woodbury_fp64(h, v, ldv, x, ldx, nrhs, T, T2)) != BEM_OK) return st;
    if (iters_out) *iters_out = 0;
    if (max_rel_resid_out) {
        double* dres = (double*)T2;     // reuse
        if ((st = residual_fp64(h, v, ldv, x, ldx, nrhs, rho, T)) != BEM_OK) return st;
        if ((st = launch_col_norm_ratio(h, rho, N, v, ldv, N, nrhs, dres)) != BEM_OK) return st;
        BEM_CUDA(h, cudaMemcpyAsync(max_rel_resid_out, dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    if (iters_out || max_rel_resid_out) return check_dev_err(h);
    return BEM_OK;
}

bem_status solve_backward(bem_handle h, const void* g_dev, int64_t ldg, void* lam_dev, int64_t ldl, int64_t nrhs) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 4) return bem_fail(h, BEM_E_INVALID, "solve_backward: call factor first");
    const int64_t N = h->N, r = h->r;
    if (!g_dev || !lam_dev || nrhs < 1 || ldg < N || ldl < N || g_dev == lam_dev)
        return bem_fail(h, BEM_E_INVALID, "solve_backward: need g, lambda (not aliased), nrhs >= 1, ld >= N");
    BEM_CUDA(h, cudaSetDevice(h->device));
    const cplx* g = (const cplx*)g_dev;
    cplx* lam = (cplx*)lam_dev;
    bem_status st;
    cplx *T = nullptr, *T2 = nullptr;
    Carve cv;
    cv.add((void**)&T, sizeof(cplx) * r * nrhs);
    cv.add((void**)&T2, sizeof(cplx) * r * nrhs);
    if ((st = cv.commit(h)) != BEM_OK) return st;
    // lambda = g/beta - beta^-2 V Kinv^H U^H g  (beta real)
    h->tag = "gemm_backward";
    if ((st = zgemm(h, OP_C, OP_N, r, nrhs, N, cmk(1, 0), h->U, N, g, ldg, cmk(0, 0), T, r)) != BEM_OK) return st;
    if ((st = zgemm(h, OP_C, OP_N, r, nrhs, r, cmk(1, 0), h->K, r, T, r, cmk(0, 0), T2, r)) != BEM_OK) return st;
    if ((st = launch_axpby(h, lam, ldl, g, ldg, cmk(1.0 / h->beta, 0), cmk(0, 0), N, nrhs)) != BEM_OK) return st;
    return zgemm(h, OP_C, OP_N, N, nrhs, r, cmk(-1.0 / (h->beta * h->beta), 0), h->Vh, r, T2, r, cmk(1, 0), lam, ldl);
}

bem_status bem_get_matrix(bem_handle h, int which, void* dst, int64_t ld) {
    if (!h || !dst) return BEM_E_INVALID;
    h->err.clear();
    BEM_CUDA(h, cudaSetDevice(h->device));
    const int64_t N = h->N;
    switch (which) {
        case BEM_MAT_S: case BEM_MAT_W: case BEM_MAT_D: {
            const cplx* src = which == BEM_MAT_S ? h->S : (which == BEM_MAT_W ? h->W : h->D);
            if (h->stage < 1 || !src) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: not assembled");
            if (ld < N) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: ld < rows");
            return launch_copy2d(h, dst, ld, src, N, N, N, sizeof(cplx));
        }
        case BEM_MAT_B:
            if (h->stage < 2) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: not filtered");
            if (ld < h->ncols) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: ld < rows");
            return launch_copy2d(h, dst, ld, h->B, h->ncols, h->ncols, N, sizeof(cplx));
        case BEM_MAT_U:
            if (h->stage < 3) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: not compressed");
            if (ld < N) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: ld < rows");
            return launch_copy2d(h, dst, ld, h->U, N, N, h->r, sizeof(cplx));
        case BEM_MAT_VH:
            if (h->stage < 3) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: not compressed");
            if (ld < h->r) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: ld < rows");
            return launch_copy2d(h, dst, ld, h->Vh, h->r, h->r, N, sizeof(cplx));
        case BEM_MAT_SIGMA:
            if (h->stage < 3) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: not compressed");
            BEM_CUDA(h, cudaMemcpyAsync(dst, h->sigma, sizeof(double) * h->ncols, cudaMemcpyDeviceToDevice, h->stream));
            return BEM_OK;
        case BEM_MAT_Q:
            if (h->stage < 2) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: not filtered");
            if (ld < N) return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: ld < rows");
            return launch_copy2d(h, dst, ld, h->Q, N, N, h->ncols, sizeof(double));
        default:
            return bem_fail(h, BEM_E_INVALID, "bem_get_matrix: unknown matrix");
    }
}

bem_status bem_timing_enable(bem_handle h, int enable) {
    if (!h) return BEM_E_INVALID;
    cudaSetDevice(h->device);
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto& r : h->trec) { h->evpool.push_back(r.a); h->evpool.push_back(r.b); }
    h->trec.clear();
    h->timing = enable != 0;
    return BEM_OK;
}

bem_status bem_timing_report(bem_handle h, char* buf, size_t len) {
    if (!h || !buf || len == 0) return BEM_E_INVALID;
    cudaSetDevice(h->device);
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<std::pair<std::string, std::pair<int, double>>> agg;
    for (auto& r : h->trec) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        bool found = false;
        for (auto& a : agg)
            if (a.first == r.name) { a.second.first += 1; a.second.second += ms; found = true; break; }
        if (!found) agg.push_back({std::string(r.name), {1, (double)ms}});
    }
    std::string s = "{";
    for (size_t i = 0; i < agg.size(); ++i) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": [%d, %.6f]", i ? ", " : "", agg[i].first.c_str(),
                 agg[i].second.first, agg[i].second.second);
        s += tmp;
    }
    s += "}";
    strncpy(buf, s.c_str(), len - 1);
    buf[len - 1] = 0;
    return BEM_OK;
}

// Far field of the current (sound-hard Green's representation): F[o, i] = C0 f_i(-xhat_o),
// C0 = e^{i pi/4} / sqrt(8 pi k), f the plane-wave right-hand side.  F is formed per call
// (N x nobs) and applied with an FP64 product.
static bem_status farfield_matrix(bem_ctx* h, const double* obs, int64_t nobs, cplx** Fm, double** ang) {
    Carve cv;
    cv.add((void**)Fm, sizeof(cplx) * h->N * nobs);
    cv.add((void**)ang, sizeof(double) * nobs);
    bem_status st = cv.commit(h);
    if (st != BEM_OK) return st;
    if ((st = launch_shift(h, obs, *ang, nobs, BEM_PI)) != BEM_OK) return st;
    return launch_rhs(h, *ang, nobs, *Fm, nullptr, h->N);
}

static cplx farfield_c0(double k) {
    const double a = 1.0 / sqrt(8.0 * BEM_PI * k);
    return cmk(a * cos(0.25 * BEM_PI), a * sin(0.25 * BEM_PI));
}

bem_status bem_farfield(bem_handle h, const double* obs_angles, int64_t nobs, const void* x, int64_t ldx,
                        int64_t nrhs, void* out, int64_t ldo) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_farfield: call bem_assemble first");
    if (!obs_angles || !x || !out || nobs < 1 || nobs > 65535 || nrhs < 1 || ldx < h->N || ldo < nobs)
        return bem_fail(h, BEM_E_INVALID, "bem_farfield: need 1 <= nobs <= 65535, nrhs >= 1, ldx >= N, ldo >= nobs");
    BEM_CUDA(h, cudaSetDevice(h->device));
    cplx* Fm = nullptr;
    double* ang = nullptr;
    bem_status st = farfield_matrix(h, obs_angles, nobs, &Fm, &ang);
    if (st != BEM_OK) return st;
    h->tag = "gemm_farfield";
    return zgemm(h, OP_T, OP_N, nobs, nrhs, h->N, farfield_c0(h->k), Fm, h->N, (const cplx*)x, ldx, cmk(0, 0),
                 (cplx*)out, ldo);
}

bem_status bem_farfield_adjoint(bem_handle h, const double* obs_angles, int64_t nobs, const void* g, int64_t ldg,
                                int64_t nrhs, void* out, int64_t ldo) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_farfield_adjoint: call bem_assemble first");
    if (!obs_angles || !g || !out || nobs < 1 || nobs > 65535 || nrhs < 1 || ldg < nobs || ldo < h->N)
        return bem_fail(h, BEM_E_INVALID,
                        "bem_farfield_adjoint: need 1 <= nobs <= 65535, nrhs >= 1, ldg >= nobs, ldo >= N");
    BEM_CUDA(h, cudaSetDevice(h->device));
    cplx* Fm = nullptr;
    double* ang = nullptr;
    bem_status st = farfield_matrix(h, obs_angles, nobs, &Fm, &ang);
    if (st != BEM_OK) return st;
    // F^H g = conj(C0) conj(Fm) g = conj( C0 Fm conj(g) ) : conjugate g into out's storage
    // is not possible (shapes differ), so go through a scratch copy of conj(g)
    cplx* gc = nullptr;
    BEM_CUDA(h, bem_dmalloc_async(h, (void**)&gc, sizeof(cplx) * nobs * nrhs));
    if ((st = launch_conj_scale(h, (const cplx*)g, ldg, gc, nobs, cmk(1, 0), nobs, nrhs)) != BEM_OK) return st;
    h->tag = "gemm_farfield_adjoint";
    st = zgemm(h, OP_N, OP_N, h->N, nrhs, nobs, farfield_c0(h->k), Fm, h->N, gc, nobs, cmk(0, 0), (cplx*)out, ldo);
    bem_dfree_async(h, gc);
    if (st != BEM_OK) return st;
    return launch_conj_scale(h, (const cplx*)out, ldo, (cplx*)out, ldo, cmk(1, 0), h->N, nrhs);
}

// Shape gradient of a far-field misfit (see bem.h).  Notation: A = I/4 + Q Q^T C_x, C_x =
// G^-1 S G^-1 N - I/4 (the filtered operator, compression taken as exact), v = G^-1 S G^-1 f,
// u = F x, x = A^-1 v, lambda = A^-H F^H gu.  With mu = Q Q^T lambda,
//   dJ = Re gu^H dF x + Re lambda^H dv - Re mu^H dC_x x
// and, writing a1 = G^-1 lambda, b1 = G^-1 f, a2 = G^-1 mu, b2 = G^-1 N x,
// a3 = G^-1 conj(S) a2, zeta = G^-1 conj(S) a1 (S is complex symmetric):
//   S terms   Re sum_ij conj(a1_i) dS_ij b1_j - conj(a2_i) dS_ij b2_j
//   N terms  -Re sum_ij conj(a3_i) dN_ij x_j
//   G terms  -Re a1^H dG v - Re zeta^H dG b1 + Re a2^H dG (G^-1 S b2) + Re a3^H dG b2
//   f terms   Re zeta^H df,   F terms  Re sum_oi (C0 sum_r x_ir conj(gu_or)) df_i(-xhat_o).
bem_status bem_shape_vjp(bem_handle h, const double* angles, const void* amplitudes, int64_t nrhs,
                         const double* obs_angles, int64_t nobs, const void* x_dev, const void* gu_dev,
                         const void* lambda_dev, double* grad_dev) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 2 || !h->S || !h->W)
        return bem_fail(h, BEM_E_INVALID, "bem_shape_vjp: needs S and N assembled and filter_apply");
    if (h->alpha != 0.0) return bem_fail(h, BEM_E_UNSUPPORTED, "bem_shape_vjp: EFIE only (alpha = 0)");
    if (h->general) return bem_fail(h, BEM_E_UNSUPPORTED, "bem_shape_vjp: equal-chord meshes only");
    if (!angles || !obs_angles || !x_dev || !gu_dev || !lambda_dev || !grad_dev || nrhs < 1 || nrhs > 65535 ||
        nobs < 1 || nobs > 65535)
        return bem_fail(h, BEM_E_INVALID, "bem_shape_vjp: bad arguments");
    BEM_CUDA(h, cudaSetDevice(h->device));
    const int64_t N = h->N, nc = h->ncols, R = nrhs;
    const cplx* x = (const cplx*)x_dev;
    const cplx* lam = (const cplx*)lambda_dev;
    const cplx* gu = (const cplx*)gu_dev;
    bem_status st;
    cplx *f, *a1, *b1, *mu, *a2, *t1, *b2, *a3, *zeta, *v, *Zx, *AB, *BB, *OmS, *OmW, *Wob, *Tq, *tmp;
    double *ang2, *sign;
    const cplx** PQ;
    Carve cv;
    for (cplx** p : {&f, &a1, &b1, &mu, &a2, &t1, &b2, &a3, &zeta, &v, &Zx, &tmp}) cv.add((void**)p, sizeof(cplx) * N * R);
    cv.add((void**)&AB, sizeof(cplx) * N * 2 * R);
    cv.add((void**)&BB, sizeof(cplx) * N * 2 * R);
    cv.add((void**)&OmS, sizeof(cplx) * N * N);
    cv.add((void**)&OmW, sizeof(cplx) * N * N);
    cv.add((void**)&Wob, sizeof(cplx) * N * nobs);
    cv.add((void**)&Tq, sizeof(cplx) * nc * R);
    cv.add((void**)&ang2, sizeof(double) * nobs);
    cv.add((void**)&sign, sizeof(double) * 4);
    cv.add((void**)&PQ, sizeof(cplx*) * 8);
    if ((st = cv.commit(h)) != BEM_OK) return st;
    BEM_CUDA(h, cudaMemsetAsync(grad_dev, 0, sizeof(double) * 2 * N, h->stream));
    // f (scaled by the amplitudes) and the G^-1 / Q Q^T / S / N products
    if ((st = launch_rhs(h, angles, R, f, nullptr, N)) != BEM_OK) return st;
    if (amplitudes) {
        if ((st = launch_scale_cols(h, f, N, (const cplx*)amplitudes, N, R)) != BEM_OK) return st;
    }
    auto ginv = [&](const cplx* in, cplx* out) { return apply_gram_inverse(h, 0, in, out, tmp, N, R, 1, N, h->hbar, false); };
    // conj(S) y = conj(S conj(y))
    auto conjS = [&](const cplx* y, cplx* out) -> bem_status {
        bem_status s2;
        if ((s2 = launch_conj_scale(h, y, N, out, N, cmk(1, 0), N, R)) != BEM_OK) return s2;
        if ((s2 = zgemm(h, OP_N, OP_N, N, R, N, cmk(1, 0), h->S, N, out, N, cmk(0, 0), t1, N)) != BEM_OK) return s2;
        return launch_conj_scale(h, t1, N, out, N, cmk(1, 0), N, R);
    };
    h->tag = "gemm_shape_vjp";
    if ((st = ginv(lam, a1)) != BEM_OK) return st;
    if ((st = ginv(f, b1)) != BEM_OK) return st;
    if ((st = dzgemm_realA(h, OP_T, nc, R, N, 1.0, h->Q, N, lam, N, 0.0, Tq, nc)) != BEM_OK) return st;
    if ((st = dzgemm_realA(h, OP_N, N, R, nc, 1.0, h->Q, N, Tq, nc, 0.0, mu, N)) != BEM_OK) return st;
    if ((st = ginv(mu, a2)) != BEM_OK) return st;
    if ((st = zgemm(h, OP_N, OP_N, N, R, N, cmk(1, 0), h->W, N, x, N, cmk(0, 0), v, N)) != BEM_OK) return st;
    if ((st = ginv(v, b2)) != BEM_OK) return st;
    if ((st = conjS(a2, Zx)) != BEM_OK) return st;                 // Zx used as scratch here
    if ((st = ginv(Zx, a3)) != BEM_OK) return st;
    if ((st = conjS(a1, Zx)) != BEM_OK) return st;
    if ((st = ginv(Zx, zeta)) != BEM_OK) return st;
    if ((st = zgemm(h, OP_N, OP_N, N, R, N, cmk(1, 0), h->S, N, b1, N, cmk(0, 0), t1, N)) != BEM_OK) return st;
    if ((st = ginv(t1, v)) != BEM_OK) return st;                   // v = G^-1 S G^-1 f
    if ((st = zgemm(h, OP_N, OP_N, N, R, N, cmk(1, 0), h->S, N, b2, N, cmk(0, 0), t1, N)) != BEM_OK) return st;
    if ((st = ginv(t1, Zx)) != BEM_OK) return st;                  // Zx = G^-1 S G^-1 N x
    // Omega^S = conj([a1 a2]) [b1 -b2]^T, Omega^W = -conj(a3) x^T, stored transposed
    if ((st = launch_copy2d(h, AB, N, a1, N, N, R, sizeof(cplx))) != BEM_OK) return st;
    if ((st = launch_copy2d(h, AB + N * R, N, a2, N, N, R, sizeof(cplx))) != BEM_OK) return st;
    if ((st = launch_copy2d(h, BB, N, b1, N, N, R, sizeof(cplx))) != BEM_OK) return st;
    if ((st = launch_axpby(h, BB + N * R, N, b2, N, cmk(-1, 0), cmk(0, 0), N, R)) != BEM_OK) return st;
    if ((st = zgemm(h, OP_N, OP_C, N, N, 2 * R, cmk(1, 0), BB, N, AB, N, cmk(0, 0), OmS, N)) != BEM_OK) return st;
    if ((st = zgemm(h, OP_N, OP_C, N, N, R, cmk(-1, 0), x, N, a3, N, cmk(0, 0), OmW, N)) != BEM_OK) return st;
    if ((st = launch_assemble_vjp(h, OmS, OmW, grad_dev)) != BEM_OK) return st;
    // Gram terms
    const cplx* hp[8] = {a1, zeta, a2, a3, v, b1, Zx, b2};
    const double hs[4] = {-1.0, -1.0, 1.0, 1.0};
    BEM_CUDA(h, cudaMemcpyAsync((void*)PQ, hp, sizeof(hp), cudaMemcpyHostToDevice, h->stream));
    BEM_CUDA(h, cudaMemcpyAsync(sign, hs, sizeof(hs), cudaMemcpyHostToDevice, h->stream));
    if ((st = launch_gram_vjp(h, (int)R, PQ, PQ + 4, sign, grad_dev)) != BEM_OK) return st;
    // right-hand sides: weights conj(zeta_iw) a_w
    if ((st = launch_conj_scale(h, zeta, N, t1, N, cmk(1, 0), N, R)) != BEM_OK) return st;
    if (amplitudes) {
        if ((st = launch_scale_cols(h, t1, N, (const cplx*)amplitudes, N, R)) != BEM_OK) return st;
    }
    if ((st = launch_rhs_vjp(h, angles, R, t1, N, grad_dev)) != BEM_OK) return st;
    // far field: weights C0 sum_r x_ir conj(gu_or) at the directions -xhat_o
    const double a0 = 1.0 / sqrt(8.0 * BEM_PI * h->k);
    const cplx c0 = cmk(a0 * cos(0.25 * BEM_PI), a0 * sin(0.25 * BEM_PI));
    if ((st = zgemm(h, OP_N, OP_C, N, nobs, R, c0, x, N, gu, nobs, cmk(0, 0), Wob, N)) != BEM_OK) return st;
    if ((st = launch_shift(h, obs_angles, ang2, nobs, BEM_PI)) != BEM_OK) return st;
    if ((st = launch_rhs_vjp(h, ang2, nobs, Wob, N, grad_dev)) != BEM_OK) return st;
    // the host copies above read hp/hs from this frame: finish before returning
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_dev_err(h);
}

bem_status bem_rhs_scale(bem_handle h, const void* v_dev, int64_t ldv, int64_t nrhs, const void* amplitudes_dev,
                         void* out_dev, int64_t ldo) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_rhs_scale: call bem_assemble first");
    if (!v_dev || !amplitudes_dev || !out_dev || nrhs < 1 || ldv < h->N || ldo < h->N)
        return bem_fail(h, BEM_E_INVALID, "bem_rhs_scale: need v, amplitudes, out, nrhs >= 1, ld >= N");
    if (out_dev == v_dev && ldo != ldv) return bem_fail(h, BEM_E_INVALID, "bem_rhs_scale: in place needs ldo == ldv");
    BEM_CUDA(h, cudaSetDevice(h->device));
    bem_status st;
    if (out_dev != v_dev)
        if ((st = launch_copy2d(h, out_dev, ldo, v_dev, ldv, h->N, nrhs, sizeof(cplx))) != BEM_OK) return st;
    return launch_scale_cols(h, (cplx*)out_dev, ldo, (const cplx*)amplitudes_dev, h->N, nrhs);
}

bem_status bem_amplitude_grad(bem_handle h, const void* v_dev, int64_t ldv, const void* lambda_dev, int64_t ldl,
                              int64_t nrhs, void* grad_dev) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_amplitude_grad: call bem_assemble first");
    if (!v_dev || !lambda_dev || !grad_dev || nrhs < 1 || ldv < h->N || ldl < h->N)
        return bem_fail(h, BEM_E_INVALID, "bem_amplitude_grad: need v, lambda, grad, nrhs >= 1, ld >= N");
    BEM_CUDA(h, cudaSetDevice(h->device));
    return launch_col_cdot(h, (const cplx*)v_dev, ldv, (const cplx*)lambda_dev, ldl, h->N, nrhs, (cplx*)grad_dev);
}

bem_status bem_shape_chain(bem_handle h, const double* tangent_dev, int64_t ncoef, const double* grad_verts_dev,
                           double* grad_coef_dev) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 1) return bem_fail(h, BEM_E_INVALID, "bem_shape_chain: call bem_assemble first");
    if (!tangent_dev || !grad_verts_dev || !grad_coef_dev || ncoef < 1 || ncoef > 65535)
        return bem_fail(h, BEM_E_INVALID, "bem_shape_chain: need tangent, gradients, 1 <= ncoef <= 65535");
    BEM_CUDA(h, cudaSetDevice(h->device));
    return launch_row_dot(h, tangent_dev, ncoef, 2 * h->N, grad_verts_dev, grad_coef_dev);
}

bem_status bem_get_info(bem_handle h, bem_info* info) {
    if (!h || !info) return BEM_E_INVALID;
    cudaSetDevice(h->device);
    BEM_CUDA(h, cudaStreamSynchronize(h->stream));
    info->N = h->N;
    info->n = h->n;
    info->r = h->r;
    info->k = h->k;
    info->h = h->hbar;
    info->alpha = h->alpha;
    info->beta = h->beta;
    info->sigma_max = h->sigma_max;
    info->stage = h->stage;
    info->prec = h->opt.prec;
    unsigned long long q = 0;
    BEM_CUDA(h, cudaMemcpy(&q, h->qpts, sizeof(q), cudaMemcpyDeviceToHost));
    info->quad_points = (int64_t)q;
    info->equal_chord = h->general ? 0 : 1;
    info->basis_block = h->general ? h->basis_block : 0;
    info->basis_iters = h->general ? h->basis_iters : 0;
    return BEM_OK;
}

}  // extern "C"
