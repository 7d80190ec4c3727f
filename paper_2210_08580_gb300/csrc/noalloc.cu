// solve_many_noalloc: the FP64 Woodbury solve of solve_many with its two r x nrhs scratch
// blocks taken from a fixed device array instead of the handle's (growable) workspace.
//
// Who needs it: callers that must not allocate device memory while they serve requests --
// code running inside CUDA stream capture, memory-capped services that reserve everything
// at start-up, or hosts embedding the library under an allocator they do not control.
// They factor once (which allocates), then solve any number of times through this call,
// which allocates nothing.
#include <cuda.h>

#include <mutex>

#include "kernels.h"

// Scratch for T = V^H v and T2 = Kinv T: two blocks of BEM_NOALLOC_MAX complex doubles
// (4 MiB each, 8 MiB in total).  Every GPU that loads the library keeps this array until
// the process exits.
#define BEM_NOALLOC_MAX (1 << 18)
static __device__ __align__(256) double2 g_noalloc_scratch[2 * BEM_NOALLOC_MAX];

static std::mutex g_noalloc_mutex;
static double2* g_noalloc_ptr[64] = {nullptr};
static unsigned long long g_noalloc_ctx[64] = {0};

typedef CUresult (*PFN_ctxGetCurrent)(CUcontext*);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long*);

// Unique id of the current context (0 when the driver cannot give one).  A device reset
// ends the context the array's address belongs to; the context created after it has a new
// id.  Caller holds g_noalloc_mutex.
static unsigned long long current_ctx_id() {
    static PFN_ctxGetCurrent get_cur = nullptr;
    static PFN_ctxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_ctxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_ctxGetId)f;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array for the current device.  In host code the array's
// name is only a host-side stand-in, so the address must come from cudaGetSymbolAddress,
// once per device and context, with that device current (a context created after a
// device reset looks it up again).
static bem_status noalloc_scratch(bem_ctx* h, double2** out) {
    if (h->device < 0 || h->device >= 64) return bem_fail(h, BEM_E_INVALID, "solve_many_noalloc: bad device");
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    const unsigned long long ctx = current_ctx_id();
    if (!g_noalloc_ptr[h->device] || (ctx != 0 && ctx != g_noalloc_ctx[h->device])) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return bem_cuda_check(h, e, "solve_many_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[h->device] = (double2*)p;
        g_noalloc_ctx[h->device] = ctx;
    }
    *out = g_noalloc_ptr[h->device];
    return BEM_OK;
}

extern "C" bem_status solve_many_noalloc(bem_handle h, const void* v_dev, int64_t ldv, void* x_dev, int64_t ldx,
                                         int64_t nrhs) {
    if (!h) return BEM_E_INVALID;
    h->err.clear();
    if (h->stage < 4) return bem_fail(h, BEM_E_INVALID, "solve_many_noalloc: call factor first");
    const int64_t N = h->N, r = h->r;
    if (!v_dev || !x_dev || nrhs < 1 || nrhs > (1 << 24) || ldv < N || ldx < N || v_dev == x_dev)
        return bem_fail(h, BEM_E_INVALID,
                        "solve_many_noalloc: need v, x (not aliased), 1 <= nrhs <= 2^24, ld >= N");
    if (r * nrhs > BEM_NOALLOC_MAX)
        return bem_fail(h, BEM_E_UNSUPPORTED,
                        "solve_many_noalloc: rank * nrhs exceeds the fixed scratch of 262144 complex "
                        "entries; split the right-hand sides into smaller batches");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return bem_cuda_check(h, e, "solve_many_noalloc: cudaSetDevice");
    double2* scratch = nullptr;
    bem_status st = noalloc_scratch(h, &scratch);
    if (st != BEM_OK) return st;
    cplx* T = scratch;                       // r x nrhs, fully overwritten (beta = 0)
    cplx* T2 = scratch + BEM_NOALLOC_MAX;    // r x nrhs, fully overwritten (beta = 0)
    const cplx* v = (const cplx*)v_dev;
    cplx* x = (cplx*)x_dev;
    // event timing may create events; keep this call free of any resource creation
    const bool timing = h->timing;
    h->timing = false;
    h->tag = "gemm_solve_noalloc";
    st = zgemm(h, OP_N, OP_N, r, nrhs, N, cmk(1, 0), h->Vh, r, v, ldv, cmk(0, 0), T, r);
    if (st == BEM_OK) st = zgemm(h, OP_N, OP_N, r, nrhs, r, cmk(1, 0), h->K, r, T, r, cmk(0, 0), T2, r);
    if (st == BEM_OK) st = launch_axpby(h, x, ldx, v, ldv, cmk(1.0 / h->beta, 0), cmk(0, 0), N, nrhs);
    if (st == BEM_OK)
        st = zgemm(h, OP_N, OP_N, N, nrhs, r, cmk(-1.0 / (h->beta * h->beta), 0), h->U, N, T2, r, cmk(1, 0), x, ldx);
    h->timing = timing;
    return st;
}
