/*
 * bem.h -- C ABI of the GB300 filtered-Calderon fast direct solver for the 2D TE-EFIE
 * (and its Yukawa-Calderon CFIE variant), after
 *   C. Henry et al., "Fast Direct Solvers for Integral Equations at Low-Frequency Based
 *   on Operator Filtering", EuCAP 2023 (arXiv 2210.08580).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the library
 *    never frees them.  Complex data are interleaved (re, im) IEEE doubles
 *    (the layout of torch.complex128 / cuDoubleComplex).
 *  - Matrices are column-major: element (i, j) of a block with leading dimension ld is at
 *    index i + j*ld.  An N x nrhs block of right-hand sides with ld = N is exactly a
 *    contiguous torch tensor of shape (nrhs, N).
 *  - A handle owns all internal matrices (S, N, D, the filtered block B, the skeleton
 *    U, V^H and the LU of the Woodbury core) and its workspace; bem_destroy frees them.
 *    Their device memory comes from the memory provider given to bem_create (the caller's
 *    allocator hooks, or the CUDA runtime).
 *    Repeating a stage on a problem of the same size reuses these allocations (a call
 *    that needs larger ones reallocates them, after synchronising the handle's stream);
 *    bem_assemble with a new N releases them first.
 *  - All work is enqueued on the handle's CUDA stream.  Calls return after enqueueing,
 *    except where a host-side result is requested (noted per call), in which case the
 *    call synchronises that stream.
 *  - The solver state advances assemble -> filter_apply -> compress_compact -> factor ->
 *    solve_many / solve_backward.  A call made out of order returns BEM_E_INVALID and
 *    changes nothing.  Re-running an earlier stage invalidates the later ones.
 *  - No call aborts, prints or exits.  On failure the status says what kind of error
 *    happened and bem_last_error(h) returns a message (valid until the next call on h).
 *  - Meshes: on an equal-chord polygon (all segment lengths equal to within 1e-10
 *    relative) the P1 Gram and Laplacian matrices are circulant and the Laplacian filter is
 *    exactly a set of Fourier modes (Sec. III-A).  Any other polygon is a non-homogeneous
 *    discretisation, for which Sec. III-A prescribes the orthonormalised Laplacian
 *    L~ = G^-1/2 L G^-1/2: G and L are then general cyclic tridiagonal matrices, solved
 *    through a bordered LDL^T factorisation, and the filter basis is computed (the lowest
 *    eigenvectors of the pencil L phi = lambda G phi, see filter_apply).  bem_shape_vjp
 *    takes equal-chord meshes only.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BEM_OK = 0,
    BEM_E_INVALID = 1,        /* bad argument or call out of order */
    BEM_E_NOMEM = 2,          /* device allocation failed */
    BEM_E_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
    BEM_E_UNSUPPORTED = 4,    /* k h too large, size limits, an equal-chord-only call */
    BEM_E_SINGULAR = 5,       /* zero pivot in the Woodbury core */
    BEM_E_NOT_CONVERGED = 6,  /* mixed-precision refinement missed refine_rtol */
    BEM_E_TIMEOUT = 7         /* a bounded device-side wait gave up */
} bem_status;

typedef enum {
    BEM_FP64 = 0,             /* every dense product in FP64 on the CUDA cores */
    BEM_MIXED_BF16 = 1        /* dense products as split-bf16 tcgen05 GEMMs (FP32 in-MMA
                                 accumulation, FP64 across K chunks) + FP64 refinement */
} bem_precision;

enum { BEM_OP_S = 1, BEM_OP_W = 2, BEM_OP_D = 4 };

/* which internal matrix bem_get_matrix copies out */
enum {
    BEM_MAT_S = 0,            /* N x N  single layer  [S]_ij = <phi_i, S phi_j>            */
    BEM_MAT_W = 1,            /* N x N  hypersingular [N]_ij = <phi_i, N phi_j> (Maue)    */
    BEM_MAT_D = 2,            /* N x N  double layer  [D]_ij = <phi_i, D phi_j>            */
    BEM_MAT_B = 3,            /* n x N  B = Q^T (C_x - alpha G^-1 D): P C_x = Q B          */
    BEM_MAT_U = 4,            /* N x r  skeleton left factor                                */
    BEM_MAT_VH = 5,           /* r x N  skeleton right factor V^H                           */
    BEM_MAT_SIGMA = 6,        /* n real doubles: singular values of the filtered compact
                                 part in the orthonormal basis, descending                 */
    BEM_MAT_Q = 7             /* N x n REAL doubles: the filter basis Q (Fourier modes on an
                                 equal-chord mesh; G-orthonormal lowest eigenvectors of the
                                 pencil (L, G) on any other mesh)                          */
};

typedef struct {
    int prec;                 /* bem_precision; default BEM_FP64 */
    int include_kernel_mode;  /* 1 (default): the filter keeps the constant Laplacian mode;
                                 0: the literal L_n^+ L_n of eq. (LapFilter), which drops it */
    double refine_rtol;       /* mixed path: target max relative residual (default 1e-10)  */
    int max_refine;           /* mixed path: maximum refinement sweeps (default 6)         */
    int split_slices;         /* mixed path: bf16 slices per operand, 0 = default (6)      */
    int rhs_slices;           /* mixed path: slices used by the right-hand-side product S Y:
                                 0 = default, one fewer than split_slices (5).  Its error (about
                                 5e-11 of max|S Y| with 5 slices) reaches the solution unrefined
                                 but far inside the mixed path's 1e-8 accuracy bar; the filter
                                 and compression products keep all slices                     */
    int solve_slices;         /* mixed path: slices used by the Woodbury solves of solve_many
                                 (the first solve and each refinement correction), 3 ..
                                 split_slices; 0 = default, all of them.  The residual
                                 products always use all slices, so fewer slices here trade
                                 a cheaper solve for refinement sweeps (about one per 2^-7
                                 digit dropped below the refine_rtol accuracy)              */
    int filter_tile_n;        /* mixed path, tile shapes of the split-bf16 products (the
                                 batching layer's tuner sets them per problem size): tile
                                 width of the filter products (112 or 128; 0 = the one that
                                 pads the filter's columns least)                           */
    int filter_split_k;       /*   K splits of the filter products (0 = the cost model's)     */
    int rhs_tile_n;           /*   tile width of the right-hand-side product (0 = automatic)  */
    int rhs_split_k;          /*   K splits of the right-hand-side product (0 = cost model)  */
    int asm_tile;             /* S/N assembly (both paths, ops without D): vertex tile edge T
                                 of one CTA, 15, 23 or 31 (0 = the default, 31).  Smaller
                                 tiles hold fewer segment pairs in shared memory, so more CTAs
                                 share an SM, at (T+1)^2/T^2 pairs per entry; any other value
                                 makes bem_create return BEM_E_INVALID                      */
} bem_options;

typedef struct {
    int64_t N;                /* unknowns (vertices = segments)                             */
    int64_t n;                /* filter modes kept (n = 2M+1 with the constant mode)        */
    int64_t r;                /* compressed rank                                            */
    double k;                 /* wavenumber                                                 */
    double h;                 /* mean chord length                                          */
    double alpha;             /* CFIE weight (0 = EFIE)                                     */
    double beta;              /* (1 + 2 alpha) / 4                                          */
    double sigma_max;         /* largest singular value of the filtered compact part        */
    int stage;                /* 0 empty, 1 assembled, 2 filtered, 3 compressed, 4 factored */
    int prec;                 /* bem_precision in use                                       */
    int64_t quad_points;      /* Gauss points (kernel evaluations) the last bem_assemble
                                 spent on separated segment pairs, counted on the device   */
    int equal_chord;          /* 1: the assembled mesh is equal-chord (circulant G, L);
                                 0: general cyclic tridiagonal G, L                        */
    int basis_block;          /* general mesh: block size p of the filter basis iteration   */
    int basis_iters;          /* general mesh: its shifted-inverse steps (0 otherwise)      */
} bem_info;

typedef struct bem_ctx* bem_handle;

/* Fills *opt with the defaults listed in bem_options. */
void bem_default_options(bem_options* opt);

/* Device memory provider of a handle: dev_alloc(bytes, alloc_ctx) returns a device pointer
 * on the handle's device (at least 256-byte aligned) or NULL when it cannot; dev_free(ptr,
 * alloc_ctx) takes it back.  The library calls them from the thread that makes the bem_* call.
 * Buffers kept across calls (the assembled matrices, B, U, V^H, the slices and workspace) are
 * freed only when the handle's stream has finished with them.  Temporaries of one call are
 * handed back as soon as the work that uses them is enqueued on the handle's stream, so the
 * provider must reuse a freed block only for work ordered after that stream's enqueued work,
 * as a stream-ordered caching allocator bound to the handle's stream does (PyTorch's, which the
 * Python binding passes by default). */
typedef void* (*bem_dev_alloc_fn)(size_t bytes, void* alloc_ctx);
typedef void (*bem_dev_free_fn)(void* ptr, void* alloc_ctx);

/* Creates a solver handle on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `opt` may be NULL (defaults).
 * dev_alloc / dev_free / alloc_ctx: the memory provider above; with both hooks every byte of
 * device memory the handle uses comes from dev_alloc and is returned through dev_free by the
 * time bem_destroy returns; with both NULL the library uses cudaMalloc / cudaMallocAsync
 * itself.  Errors: BEM_E_INVALID (NULL h, exactly one hook NULL, bad options or device),
 * BEM_E_NOMEM, BEM_E_CUDA. */
bem_status bem_create(bem_handle* h, int device, void* cuda_stream, const bem_options* opt,
                      bem_dev_alloc_fn dev_alloc, bem_dev_free_fn dev_free, void* alloc_ctx);

/* Frees everything the handle owns (synchronises its stream first).  NULL is accepted. */
bem_status bem_destroy(bem_handle h);

/* Message of the last failed call on h (empty string if none). */
const char* bem_last_error(bem_handle h);

/* Redirects subsequent work to another stream. */
bem_status bem_set_stream(bem_handle h, void* cuda_stream);

/* bem_assemble -- dense Galerkin matrices of the single-layer S, hypersingular N and
 * double-layer D operators of Sec. II,
 *     [X]_ij = <phi_i, X phi_j>,  g2(r) = (i/4) H0^(1)(k r),
 * on the closed polygon with N vertices verts_xy_dev[2*i], verts_xy_dev[2*i+1]
 * (counter-clockwise, segment i joins vertex i to vertex i+1 mod N, P1 hats phi_i).
 * N uses Maue's integration by parts:
 *     <phi_i, N phi_j> = int int g2 [phi_i' phi_j' - k^2 (nu_x . nu_y) phi_i phi_j].
 * `ops` is a mask of BEM_OP_S | BEM_OP_W | BEM_OP_D; S and W are needed by the EFIE
 * path, D by the CFIE (alpha != 0).  Requires N >= 16, k > 0, k*h <= 2 for the longest
 * chord h.  Chords that differ by more than 1e-10 of their mean make the mesh a general
 * one (see the notes at the top): its Gram matrix is factored here.  Synchronises the
 * stream once (to validate the mesh).  Errors: BEM_E_INVALID (bad arguments),
 * BEM_E_UNSUPPORTED (k h > 2), BEM_E_NOMEM, BEM_E_CUDA. */
bem_status bem_assemble(bem_handle h, const double* verts_xy_dev, int64_t N, double k,
                        unsigned ops);

/* bem_assemble_batch -- bem_assemble (S and N) for nprob independent problems at once: handle
 * hs[q] (all on one device, each its own stream and options, none twice) assembles the polygon
 * verts_dev[q] (2 Ns[q] device doubles) at wavenumber ks[q] (host arrays of nprob pointers /
 * values).  The checks and the per-problem preparation run as in bem_assemble (one stream sync
 * per problem for the mesh check); the tiles of all problems then run in ONE persistent launch
 * on hs[0]'s stream, CTAs taking tiles from a global queue (largest problems first), so that
 * small problems fill the GPU beside large ones; each handle's stream waits for that launch
 * before its own later work.  Synchronises hs[0]'s stream.  The batching layer's assembly
 * stage; the paper solves one problem at a time.  Errors as bem_assemble (the message of a
 * failing problem q > 0 is also left on hs[0]). */
bem_status bem_assemble_batch(bem_handle* hs, int64_t nprob, const double* const* verts_dev, const int64_t* Ns,
                              const double* ks);

/* filter_apply -- the Laplacian filter of eq. (LapFilter) applied to the compact part of
 * the Calderon-preconditioned equation (Sec. IV-A).  With the equal-chord mesh the filter
 * is P = Q Q^T, Q the N x n real Fourier modes |m| <= M (n = 2M+1; columns ordered
 * constant, cos 1, sin 1, cos 2, sin 2, ...).  Computes the n x N block
 *     B = Q^T (G^-1 S G^-1 N - I/4 - alpha G^-1 D)
 *       = diag(1/g_m) (Q^T S G^-1 N - alpha Q^T D) - Q^T/4,
 * so that the filtered operator in nodal coordinates is beta I + Q B with
 * beta = (1 + 2 alpha)/4 (alpha = 0: filtered TE-EFIE; alpha > 0: filtered Yukawa-Calderon
 * TE-CFIE).  On any other mesh Q is the G-orthonormal basis of the n lowest eigenvectors of
 * the pencil L phi = lambda G phi (Q = G^-1/2 V_n, V_n those of L~; the filter in nodal
 * coordinates is Q Q^T G), g_m = 1, and
 *     B = Q^T G (G^-1 S G^-1 N - I/4 - alpha G^-1 D) = (Q^T S) G^-1 N - alpha Q^T D - (G Q)^T/4;
 * Q comes from Chebyshev-accelerated shift-and-invert subspace iteration on
 * sigma (L + sigma G)^-1 G (a block of about 1.5 n + 9 columns, at most 1023, started from
 * arclength Fourier modes, Cholesky-QR G-orthonormalised) and one Rayleigh-Ritz step through
 * the Jacobi SVD; its span matches the eigenvectors to rounding (a non-positive Cholesky
 * pivot returns BEM_E_SINGULAR).
 * n_modes must be odd, 3 <= n_modes <= min(N - 1, 1023).  Needs S, W (and D if alpha != 0). */
bem_status filter_apply(bem_handle h, int64_t n_modes, double alpha);

/* compress_compact -- skeleton of the filtered compact part (Sec. IV-C): computes the SVD
 * of diag(sqrt g) B G^-1/2 (the block in the orthonormal, G^1/2-weighted basis of the
 * paper; G^-1/2 is taken as F^-1 with F^T F = G, which leaves the singular values and left
 * singular vectors unchanged) by Householder QR plus one-sided Jacobi, keeps the singular values
 * sigma_i >= rel_tol * sigma_1 and forms U (N x r), V^H (r x N) with Q B ~= U V^H.
 * Writes the rank to *rank_out (host pointer, may be NULL); synchronises the stream. */
bem_status compress_compact(bem_handle h, double rel_tol, int64_t* rank_out);

/* factor -- Woodbury core of (beta I + U V^H)^-1 (Sec. IV-C): K = I_r + beta^-1 V^H U and
 * its LU factorisation with partial pivoting.  Errors: BEM_E_SINGULAR if a pivot is zero
 * (reported when solve_many is next called, or here if the stream is synchronised). */
bem_status factor(bem_handle h);

/* bem_rhs_planewave -- right-hand sides for incident plane waves u_inc = exp(i k d.x),
 * d = (cos a_w, sin a_w), a_w = angles_dev[w] (device doubles):
 *     f_i = -<phi_i, d u_inc / d nu>               (the TE-EFIE data times i k, Sec. II)
 *     v   = G^-1 S G^-1 f - alpha G^-1 h2,  [h2]_i = <phi_i, u_inc>
 * (v is the right-hand side of beta x + Q B x = v in nodal coordinates).  f_out and v_out
 * are N x nrhs complex blocks with leading dimension ld >= N; either may be NULL;
 * 1 <= nrhs <= 65535.
 * Needs bem_assemble (S); alpha is the value given to filter_apply (0 before). */
bem_status bem_rhs_planewave(bem_handle h, const double* angles_dev, int64_t nrhs,
                             void* f_out_dev, void* v_out_dev, int64_t ld);

/* bem_rhs_pointsource -- right-hand sides for line sources: the incident field of source w is
 * the 2D free-space field u_inc(x) = g2(|x - r0_w|) = (i/4) H0^(1)(k |x - r0_w|) (the "dipole"
 * source of Sec. V, read as a z-directed line source, which radiates a TE field H_z = u_inc),
 * r0_w = (src_xy_dev[2w], src_xy_dev[2w+1]) (device doubles), off the curve:
 *     f_i = -<phi_i, d u_inc / d nu>,   v = G^-1 S G^-1 f - alpha G^-1 h2,  [h2]_i = <phi_i, u_inc>,
 * as bem_rhs_planewave for plane waves (8-point Gauss-Legendre per segment, FP64).  f_out,
 * v_out: N x nsrc blocks (ld >= N), either may be NULL; 1 <= nsrc <= 65535.  The sources
 * must lie at a distance of several chords from the curve (the rule is exact to rounding for
 * distances above about 4 h).  Needs bem_assemble. */
bem_status bem_rhs_pointsource(bem_handle h, const double* src_xy_dev, int64_t nsrc, void* f_out_dev,
                               void* v_out_dev, int64_t ld);

/* bem_factor_rhs_planewave -- compress_compact(rel_tol), factor and bem_rhs_planewave in one
 * call (Sec. IV-C and Sec. II), with the same results: once the compression's QR has run,
 * the right-hand sides (their product with S is the largest of the path) run on a second
 * stream of the handle while the rest of the compression and the factor run on a third, of
 * the highest priority; both are joined to the handle's stream before the call returns.
 * The handle keeps the two streams until bem_destroy.  Arguments as
 * for those calls; v_out_dev is required (f_out_dev may be NULL).  Needs filter_apply.
 * Writes the rank to *rank_out; synchronises the handle's stream as compress_compact does.
 * Errors: those of the three calls (the first one met is returned). */
bem_status bem_factor_rhs_planewave(bem_handle h, double rel_tol, const double* angles_dev, int64_t nrhs,
                                    void* f_out_dev, void* v_out_dev, int64_t ld, int64_t* rank_out);

/* solve_many -- x = (beta I + U V^H)^-1 v by the Woodbury identity (Sec. IV-C):
 *     x = v/beta - beta^-2 U (I_r + beta^-1 V^H U)^-1 V^H v,
 * for nrhs columns v (ldv >= N) into x (ldx >= N).  x may not alias v.
 * In BEM_MIXED_BF16 mode the products run as split-bf16 tensor-core GEMMs and the
 * result is refined against the FP64 residual v - (beta x + U V^H x) until its max
 * relative column norm is <= refine_rtol.  iters_out (host, may be NULL) receives the
 * refinement sweeps used; max_rel_resid_out (host, may be NULL) the max relative residual.
 * If either pointer is non-NULL the call synchronises the stream.
 * Errors: BEM_E_NOT_CONVERGED (x holds the best iterate), BEM_E_SINGULAR. */
bem_status solve_many(bem_handle h, const void* v_dev, int64_t ldv, void* x_dev, int64_t ldx,
                      int64_t nrhs, int32_t* iters_out, double* max_rel_resid_out);

/* solve_backward -- adjoint solve (beta I + U V^H)^H lambda = g, i.e.
 *     lambda = g/conj(beta) - conj(beta)^-2 V (I_r + conj(beta)^-1 U^H V)^-1 U^H g,
 * which gives dJ/dv = lambda for a real loss J of x (the Woodbury identity applied to the
 * adjoint operator).  Same layouts as solve_many; lambda may not alias g. */
bem_status solve_backward(bem_handle h, const void* g_dev, int64_t ldg, void* lambda_dev,
                          int64_t ldl, int64_t nrhs);

/* solve_many_noalloc -- the paper has no counterpart to this call; it exists for callers
 * that cannot allocate device memory while they solve: code recorded inside CUDA stream
 * capture, services that reserve all of their memory at start-up, or hosts that embed the
 * library under an allocator they do not own.  It computes the same FP64 Woodbury solve as
 * solve_many's FP64 path, x = v/beta - beta^-2 U (I_r + beta^-1 V^H U)^-1 V^H v, but takes
 * its two r x nrhs scratch blocks from a fixed array compiled into the library instead of
 * the handle's workspace, and calls no allocator.
 *  - Limit: r * nrhs <= 262144 (the array holds 2 x 262144 complex doubles, 8 MiB, which
 *    every GPU that loads the library keeps until the process exits); larger requests
 *    return BEM_E_UNSUPPORTED without doing any work.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *    make that first call before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents (nothing in it
 *    needs to start at zero).  Calls whose work overlaps on the GPU -- two streams, or two
 *    handles -- race on the array: serialise them.
 *  - Layouts, aliasing rules and the limit 1 <= nrhs <= 2^24 are those of solve_many; no
 *    refinement and no residual report (use solve_many for those).  Needs factor.
 *  - On a BEM_MIXED_BF16 handle it solves with the factors that handle built (U, V^H and
 *    the core from tensor-core products) in FP64, without refinement: the result is the
 *    exact inverse of that handle's compressed operator up to FP64 rounding, which is what
 *    solve_many's refinement converges to. */
bem_status solve_many_noalloc(bem_handle h, const void* v_dev, int64_t ldv, void* x_dev, int64_t ldx,
                              int64_t nrhs);

/* bem_solve_batch -- the FP64 Woodbury solve of solve_many (Sec. IV-C: x = v/beta -
 * beta^-2 U (I_r + beta^-1 V^H U)^-1 V^H v) for nprob factored problems in ONE persistent
 * launch: problem q solves with handle hs[q] the nrhs[q] right-hand sides v_dev[q] (column-major
 * N_q x nrhs[q] complex128, leading dimension ldv[q]) into x_dev[q] (ldx[q]).  The arrays are
 * host arrays of nprob entries; the buffers are device memory the caller owns.  CTAs take
 * 64 x 64 tiles of all problems' products from one global queue (V^H v in slices of N, 256
 * long up to N = 16384 and at most 64 per problem beyond, then the core product, then x), so small problems fill the GPU beside large ones;
 * a tile that needs another stage's results waits for them with a bounded device-side wait.
 * Runs on hs[0]'s stream after every handle's earlier work; every handle's later work waits
 * for it.  Synchronises hs[0]'s stream (to read the device status).  Scratch: the core
 * products, sum over q of r_q nrhs[q] (s_q + 1) complex doubles, s_q = min(ceil(N_q / 256), 64)
 * slices (up to 65 r_q nrhs[q]), taken from
 * hs[0]'s device memory provider for the call.  The same handle may appear more than once;
 * no x_dev[q] may overlap any v_dev or another x_dev.  On a BEM_MIXED_BF16 handle it solves
 * with that handle's factors in FP64 without refinement, as solve_many_noalloc does.  The
 * batching layer's solve stage; the paper solves one problem at a time.
 * Errors: BEM_E_INVALID (null arrays, nprob outside [1, 65536], a handle not factored or on
 * another device, bad v/x/ld/nrhs; the message names the problem and is left on hs[0]),
 * BEM_E_UNSUPPORTED (N >= 2^30), BEM_E_NOMEM/BEM_E_CUDA (scratch, launch), BEM_E_TIMEOUT
 * (a device-side wait gave up, after 10 s; x is then incomplete). */
bem_status bem_solve_batch(bem_handle* hs, int64_t nprob, const void* const* v_dev, const int64_t* ldv,
                           void* const* x_dev, const int64_t* ldx, const int64_t* nrhs);

/* bem_solve_batch_stall_check -- failure detection of bem_solve_batch's device-side waits,
 * without a GPU fault: the same call and kernel, but the first completion counter of the
 * first problem in the queue starts far below its target, so the tiles waiting on it give up
 * after stall_ms (1 .. 10000) of wall time instead of the production limit of 10 s.  Expected
 * result: BEM_E_TIMEOUT, with x incomplete, the device status word cleared and the handles
 * usable for the next call.  Other errors as bem_solve_batch.  No paper counterpart. */
bem_status bem_solve_batch_stall_check(bem_handle* hs, int64_t nprob, const void* const* v_dev,
                                       const int64_t* ldv, void* const* x_dev, const int64_t* ldx,
                                       const int64_t* nrhs, int stall_ms);

/* bem_farfield -- far field of the current x (P1 coefficients, x = -u_tot on the curve)
 * for the sound-hard problem of Sec. II: Green's representation u_s = int u_tot dg/dnu_y,
 * and g(x, y) ~ C0 e^{ik|x|}/sqrt|x| e^{-ik xhat.y}, C0 = e^{i pi/4}/sqrt(8 pi k), give
 *     u_inf(xhat_o) = sum_i F[o, i] x_i,  F[o, i] = i k C0 <phi_i, (xhat_o.nu) e^{-ik xhat_o.y}>,
 * xhat_o = (cos b_o, sin b_o), b_o = obs_angles_dev[o].  x: N x nrhs (ldx >= N); out:
 * nobs x nrhs (ldo >= nobs), complex, column-major, device.  1 <= nobs <= 65535.
 * The paper states no far field; it is the observable of the differentiation layer.
 * Needs bem_assemble.  Errors: BEM_E_INVALID. */
bem_status bem_farfield(bem_handle h, const double* obs_angles_dev, int64_t nobs, const void* x_dev,
                        int64_t ldx, int64_t nrhs, void* out_dev, int64_t ldo);

/* bem_farfield_adjoint -- out = F^H g for g: nobs x nrhs (ldg >= nobs) into out: N x nrhs
 * (ldo >= N), the vector-Jacobian product of bem_farfield (with solve_backward it gives the
 * gradient of a far-field misfit with respect to the right-hand side). */
bem_status bem_farfield_adjoint(bem_handle h, const double* obs_angles_dev, int64_t nobs, const void* g_dev,
                                int64_t ldg, int64_t nrhs, void* out_dev, int64_t ldo);

/* bem_shape_vjp -- gradient with respect to the vertex coordinates of a real far-field
 * misfit J(u), u = F x, x = A^-1 (a_w v_w): the adjoint (reverse) derivative through the
 * assembly of S and N (every segment pair's integrals differentiated: the Gauss rule of
 * separated pairs, the closed forms of self and adjacent pairs), the Gram matrix, the
 * plane-wave right-hand sides and the far-field operator.  A = I/4 + Q Q^T C_x is the
 * filtered operator of Sec. IV-A with the compression taken as exact (use compress_compact
 * with rel_tol = 0), Q the Fourier filter basis (fixed for equal-chord meshes), so the
 * result is the gradient along equal-chord deformations.  Inputs (device): angles (nrhs
 * incidence angles of the right-hand sides), amplitudes (nrhs complex a_w, NULL = all 1),
 * obs_angles (nobs), x (N x nrhs, the solution), gu (nobs x nrhs: dJ/du in the
 * dJ/dRe + i dJ/dIm convention), lambda = A^-H F^H gu (N x nrhs, from bem_farfield_adjoint
 * and solve_backward).  Output: grad (2N doubles, (x_i, y_i), overwritten).  EFIE only
 * (alpha = 0), N >= 5, FP64 arithmetic; synchronises the stream.  The paper states no
 * derivative; this is the differentiation layer's shape derivative. */
bem_status bem_shape_vjp(bem_handle h, const double* angles_dev, const void* amplitudes_dev, int64_t nrhs,
                         const double* obs_angles_dev, int64_t nobs, const void* x_dev, const void* gu_dev,
                         const void* lambda_dev, double* grad_dev);

/* bem_rhs_scale -- right-hand sides of incident fields with complex amplitudes: out[:, w] =
 * a_w v[:, w] for the N x nrhs block v (ldv >= N) and nrhs complex amplitudes a (device);
 * out (ldo >= N) may be v itself (then ldo == ldv).  The paper states the incident field with
 * unit amplitude; this is the forward map of the amplitude derivative below. */
bem_status bem_rhs_scale(bem_handle h, const void* v_dev, int64_t ldv, int64_t nrhs, const void* amplitudes_dev,
                         void* out_dev, int64_t ldo);

/* bem_amplitude_grad -- gradient of a real misfit J with respect to the complex amplitudes a_w
 * of the right-hand sides a_w v_w, given lambda = A^-H (dJ/dx) (solve_backward):
 *     grad[w] = v[:, w]^H lambda[:, w]     (the dJ/dRe a + i dJ/dIm a convention)
 * v, lambda: N x nrhs (ld >= N), device; grad: nrhs complex, device.  Fixed-order sums. */
bem_status bem_amplitude_grad(bem_handle h, const void* v_dev, int64_t ldv, const void* lambda_dev, int64_t ldl,
                              int64_t nrhs, void* grad_dev);

/* bem_shape_chain -- chain rule from the vertex gradient to curve parameters p_c:
 *     grad_coef[c] = sum_{i, d} tangent[c][i][d] grad_verts[i][d],  tangent[c][i][d] = d r_i,d / d p_c
 * tangent: ncoef x N x 2 doubles (row-major, device; for equal-chord meshes the implicit
 * derivative of the mesh), grad_verts: N x 2 (bem_shape_vjp), grad_coef: ncoef doubles. */
bem_status bem_shape_chain(bem_handle h, const double* tangent_dev, int64_t ncoef, const double* grad_verts_dev,
                           double* grad_coef_dev);

/* Copies an internal matrix (BEM_MAT_*) into dst_dev with leading dimension ld (>= rows).
 * For BEM_MAT_SIGMA, dst_dev receives n doubles and ld is ignored. */
bem_status bem_get_matrix(bem_handle h, int which, void* dst_dev, int64_t ld);

/* Sizes and scalars of the current state (synchronises the stream). */
bem_status bem_get_info(bem_handle h, bem_info* info);

/* Profiling support (not part of the method).  While enabled, every kernel launch of the
 * handle is bracketed by CUDA events recorded on the handle's stream; enabling clears the
 * records.  bem_timing_report synchronises the stream and writes a JSON object
 * {"<kernel or GEMM call site>": [launches, total_ms], ...} into buf (NUL-terminated,
 * truncated to len).  Returns BEM_E_INVALID on a NULL handle or buffer. */
bem_status bem_timing_enable(bem_handle h, int enable);
bem_status bem_timing_report(bem_handle h, char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* BEM_GB300_H */
