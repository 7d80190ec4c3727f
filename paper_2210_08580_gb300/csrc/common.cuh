// Shared device/host helpers of the GB300 BEM library: complex arithmetic on double2,
// launch checking, a bounded grid-wide barrier for cooperative kernels, and the handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/bem.h"

#ifndef BEM_PI
#define BEM_PI 3.14159265358979323846
#endif

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmk(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfma_conj(cplx& acc, cplx a, cplx b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    double d = 1.0 / cabs2(b);
    return cmk((a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d);
}

// Device-side status word: kernels OR error bits into it instead of trapping.
enum { DEVERR_TIMEOUT = 1, DEVERR_SINGULAR = 2, DEVERR_BOUNDS = 4, DEVERR_NAN = 8 };

// Bounded grid barrier for kernels launched with cudaLaunchCooperativeKernel (all CTAs
// co-resident).  `bar[0]` counts the arrivals of the launch.  A CTA that waits
// longer than the spin limit sets DEVERR_TIMEOUT in *err and returns false; callers then
// return, so every CTA ends (the others time out as well).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err) {
    // bar[0] counts arrivals over the whole launch (zeroed before it): the CTAs of barrier g
    // are through once the count reaches (g + 1) nblocks, so the last arrival releases the
    // others by its own increment (no reset, no second word on the critical path)
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();                                   // this CTA's writes before its arrival
        const unsigned arrived = atomicAdd(bar, 1u);
        const unsigned target = (arrived / nblocks + 1) * nblocks;
        volatile unsigned* vcount = bar;
        long long spins = 0;
        while ((int)(*vcount - target) < 0) {
            if (++spins > (1ll << 26)) { atomicOr(err, DEVERR_TIMEOUT); ok = 0; break; }
            if ((spins & 1023) == 0 && *(volatile int*)err) { ok = 0; break; }
            if (spins > 64) __nanosleep(64);
        }
        __threadfence();                                   // the others' writes after it
        if (*(volatile int*)err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct bem_ctx {
    int device = 0;
    cudaStream_t stream = 0;
    bem_options opt{};
    std::string err;

    // device memory provider: the caller's hooks (bem_create), or the CUDA runtime when NULL
    void* (*dev_alloc)(size_t, void*) = nullptr;
    void (*dev_free)(void*, void*) = nullptr;
    void* alloc_ctx = nullptr;
    double* btab = nullptr;           // far-field Bessel tables (this handle's copy)
    float4* btabf = nullptr;

    // geometry and assembly
    int64_t N = 0;
    double k = 0.0, hbar = 0.0;
    double hmax = 0.0;                // longest chord
    bool general = false;             // chords not equal (spread above 1e-10 of the mean):
                                      // general cyclic tridiagonal G and L (mesh.cu)
    int basis_block = 0, basis_iters = 0;   // subspace iteration of the last general filter basis
    double* gfac = nullptr;           // bordered LDL^T of the general Gram matrix and the chunk
                                      // propagators of its solves (mesh.cu)
    unsigned ops = 0;
    double* seg = nullptr;            // 5*N: x0, y0, tx, ty, h (SoA)
    cplx *S = nullptr, *W = nullptr, *D = nullptr;
    int* rexp = nullptr;              // 2N: largest IEEE exponent field per column of S, W (W
                                      // without its near band), taken during the assembly
    bool rexp_valid = false;          // rexp belongs to the S, W now held
    cplx* k1 = nullptr;               // N: row sums of N (its k^2 term's, exact in Maue's form)
    double2* kpart = nullptr;         // per-tile partials of k1 (tile slots x N)
    int64_t kpart_slots = 0;          // tile slots kpart holds
    bool k1_valid = false;            // k1 belongs to the N now held
    std::map<void**, size_t> caps;   // bytes allocated behind each stage buffer (reused while large enough)

    // filter
    int64_t n = 0, M = 0, ncols = 0;  // n modes requested, ncols Fourier columns kept
    double alpha = 0.0, beta = 0.25;
    cplx* B = nullptr;                // ncols x N, ld = ncols
    cplx* Bs = nullptr;               // diag(sqrt g) B
    double* gm = nullptr;             // ncols Gram eigenvalues of the Fourier columns (1 on a
                                      // general mesh, whose basis is G-orthonormal)
    double* Q = nullptr;              // N x ncols filter basis: Fourier modes, or on a general
                                      // mesh the lowest eigenvectors of the pencil (L, G)
    double* GQ = nullptr;             // N x ncols: G Q (general mesh only)

    // compression / factor
    int64_t r = 0;
    double sigma_max = 0.0;
    double* sigma = nullptr;          // n
    cplx* E = nullptr;                // n x n right singular vectors (ld = n), sorted
    cplx *U = nullptr, *Vh = nullptr; // N x r (ld N), r x N (ld r)
    cplx* K = nullptr;                // r x r inverse of the Woodbury core (ld r)
    int* piv = nullptr;               // r

    // workspace
    void* work = nullptr;
    size_t work_bytes = 0;
    // bem_factor_rhs_planewave: the right-hand sides run on aux beside the compression and
    // the factor; while they are enqueued (rhs_aux), their scratch comes from work2 and the
    // split products' B operand from its own buffer, so nothing is shared with the other chain
    cudaStream_t aux = nullptr;
    cudaStream_t hi = nullptr;       // the compression and factor meanwhile, at the highest
                                     // priority: the block scheduler serves its kernels before
                                     // the GEMM's queued CTAs (at equal priority it would not
                                     // start them until the GEMM's last CTAs were dispatched)
    void* work2 = nullptr;
    size_t work2_bytes = 0;
    bool rhs_aux = false;
    int* dev_err = nullptr;           // device status word
    unsigned* bar = nullptr;          // grid barrier words (2)
    unsigned long long* qpts = nullptr;   // Gauss points of separated pairs, last assembly
    int stage = 0;

    // mixed-precision state (owned by the tensor-core module)
    void* tc = nullptr;

    // optional per-launch timing (CUDA events on the handle's stream)
    bool timing = false;
    const char* tag = "kernel";       // label of the next timed GEMM call site
    struct TimingRec { const char* name; cudaEvent_t a, b; };
    std::vector<TimingRec> trec;
    std::vector<cudaEvent_t> evpool;
};

cudaEvent_t bem_event_get(bem_ctx* h);
// Brackets the launch statement(s) with events when timing is enabled.
#define BEM_TIMED(h, name, ...)                                                  \
    do {                                                                         \
        cudaEvent_t _ta = nullptr;                                               \
        if ((h)->timing) { _ta = bem_event_get(h); cudaEventRecord(_ta, (h)->stream); } \
        __VA_ARGS__;                                                             \
        if ((h)->timing) {                                                       \
            cudaEvent_t _tb = bem_event_get(h);                                  \
            cudaEventRecord(_tb, (h)->stream);                                   \
            (h)->trec.push_back({(name), _ta, _tb});                             \
        }                                                                        \
    } while (0)

// error helpers ---------------------------------------------------------------------------
bem_status bem_fail(bem_ctx* h, bem_status st, const std::string& msg);
bem_status bem_cuda_check(bem_ctx* h, cudaError_t e, const char* what);
#define BEM_CUDA(h, call)                                                       \
    do {                                                                        \
        cudaError_t _e = (call);                                                \
        if (_e != cudaSuccess) return bem_cuda_check((h), _e, #call);           \
    } while (0)
#define BEM_LAUNCH(h, what)                                                     \
    do {                                                                        \
        cudaError_t _e = cudaGetLastError();                                    \
        if (_e != cudaSuccess) return bem_cuda_check((h), _e, what);            \
    } while (0)

// workspace: returns a device pointer of at least `bytes`, growing the handle's buffer
bem_status bem_workspace(bem_ctx* h, size_t bytes, void** out);   // work2 while rhs_aux is set

// Device memory of a handle.  With the caller's hooks (bem_create) every byte comes from
// dev_alloc and goes back through dev_free; without them from the CUDA runtime.
// bem_dmalloc/bem_dfree: buffers kept across calls (freed only after the stream is idle).
// bem_dmalloc_async/bem_dfree_async: stream-ordered temporaries of one call on h->stream
// (cudaMallocAsync/cudaFreeAsync; with hooks, dev_free is called once the work using the
// block is enqueued, and the provider must order reuse after it, as a stream-ordered
// caching allocator on that stream does).  A failed allocation is cudaErrorMemoryAllocation.
cudaError_t bem_dmalloc(bem_ctx* h, void** p, size_t bytes);
void bem_dfree(bem_ctx* h, void* p);
cudaError_t bem_dmalloc_async(bem_ctx* h, void** p, size_t bytes);
void bem_dfree_async(bem_ctx* h, void* p);
