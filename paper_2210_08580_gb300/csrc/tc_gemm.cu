// Mixed-precision dense products on the GB300 tensor cores (tcgen05, TMEM, TMA).
//
// A complex product C = A B (A: M x K, B: K x m, FP64) is evaluated as one real GEMM of
// planar part matrices: a complex row i of A becomes part rows 2i (Re) and 2i+1 (Im), a
// complex column j of B part columns 2j (Re) and 2j+1 (Im); a real operand keeps one part.
// The GEMM C' = A' B' then holds Re A Re B, Re A Im B, Im A Re B and Im A Im B in adjacent
// rows and columns, and the epilogue forms Re C = RR - II, Im C = RI + IR (or takes the two
// parts directly when one operand is real, which halves the work).
//
// Each operand is split into S bf16 slices (error-free splitting after Ozaki et al.,
// Numer. Algorithms 2012): with a power-of-two scale per row of A' (2^e_i) and per column
// of B (2^f_j, shared by the parts), x 2^-e = sum_s a_s 2^{-7(s+1)} with integers |a_0| <= 128, |a_s| <= 64;
// slice s is stored pre-multiplied by 2^{-7s}, which bf16 holds exactly.  Products of
// slices (s, t) with s + t <= S - 1 are accumulated by tcgen05.mma (kind::f16, FP32
// accumulation) into four TMEM accumulators: d = 0, 1, 2 and d >= 3 (d = s + t).  Over a
// K' chunk of 512 the d = 0, 1, 2 sums are multiples of 2^-7d below 2^24 of that unit
// (|d0 e0| <= 2^14, |d0 e1| + |d1 e0| <= 2^14, the three d = 2 products <= 2^14 + 2^12 per
// k), so FP32 accumulation is exact for them (measured on GB300: a group of one magnitude
// is exact, while mixing groups 7 or more bits apart in one accumulator rounds at 2^-24 of
// it); the d >= 3 sum carries that 2^-24 rounding on a term 2^-21 below the leading one.
// After each chunk the epilogue warps add the accumulators into double-float (hi, lo)
// registers; the result is rescaled by 2^{e_i + f_j - 14} and written in FP64.
//
// Kernel: one 128 x BN tile of C' per CTA, BN = 128, or 112 when that pads the B part rows
// less (the filter's 201 and 402 columns), split over K' when that fills the GPU better;
// 10 warps: warp 0 issues TMA loads (3D tensor
// maps over the stacked slices, 64-byte swizzle, 32-element K blocks, 2 stages), warp 1
// allocates TMEM and issues the MMAs (S is a template parameter, so the S(S+1)/2 x 2 MMAs
// of a K block are one straight-line sequence with constant descriptor offsets: a loop
// that rebuilt descriptors per MMA issued slower than the tensor pipe executes), warps
// 2..9 drain TMEM (2 warps per TMEM lane quarter, 64 and BN - 64 columns).  Every mbarrier wait is
// bounded; a timeout sets the handle's device error word and the CTA winds down, freeing
// its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "dfloat.cuh"
#include "kernels.h"
#include "tc_gemm.h"

#define TC_BM 128
#define TC_BN 128                   // tile width (B part rows); 112 where it pads less (201, 402)
#define TC_BK 32
#define TC_STAGES 2
#define TC_CHUNK_KB 16              // K' chunk of 16 x 32 = 512 between TMEM flushes
#define TC_NACC 4                   // TMEM accumulators (4 x 128 columns = all 512)
#define TC_SMAX 7
#define TC_TILE_BYTES (TC_BM * TC_BK * 2)          // 8 KiB per slice tile (A and B alike)
#define TC_STASH_BYTES (TC_BM * (TC_BN + 1) * 8)   // epilogue staging of (hi, lo) pairs
#define TC_THREADS 320             // 10 warps: TMA, MMA, 8 epilogue

// ------------------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok;
}
// bounded wait: false (and DEVERR_TIMEOUT set) if the phase does not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && *(volatile int*)err) return false;
    }
    atomicOr(err, DEVERR_TIMEOUT);
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor, K-major operand tile with 64-byte swizzle: rows of
// 64 B (32 bf16), 8-row groups 512 B apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

struct TcGemmArgs {
    int M, Ncols;            // rows of the A and B part matrices (tiles run over these)
    int Ml, ml;              // logical rows / columns of the complex result
    int aC, bC;              // A / B complex (two part rows each) or real
    int nkb;                 // K' blocks of 32
    int S;                   // slices per operand
    const int* ea;           // M row exponents
    const int* eb;           // Ncols column exponents
    double2* out;            // complex output
    int64_t ldo;
    int transposed;          // 0: out[i + j ldo], 1: out[j + i ldo]
    double alpha, beta;      // out = alpha C + beta out
    int* err;
    int kps;                 // K' blocks per split (blockIdx.y); == nkb without split
    double2* part;           // split partials [split][j][i] (M x m each), or null
    // blocked products (zmode 1): A and B hold real row blocks (Re, Im, Re + Im of a complex
    // operand, or one real block); product z = blockIdx.z multiplies row block zA[z] of A
    // by row block zB[z] of B (rows per block Ml and ml) and writes its real result, scaled,
    // to outr[((z splits + split) ml + j) Ml + i]; the caller combines the products
    int zmode;
    int zA[3], zB[3];
    double* outr;
};

template <int S, int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcGemmArgs p) {
    static_assert(BN == 128 || BN == 112, "tile width");
    // a B slice tile fills BN rows of its 8 KiB slot (the descriptors' offsets stay those
    // of 128-row tiles); the MMA's N and the accumulators' column stride are BN
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // layout: [stage][A slices][B slices] tiles (reused as the epilogue stash once the
    // MMAs are done), then the barriers after max(stages, stash)
    const size_t stage_bytes = (size_t)2 * S * TC_TILE_BYTES;
    const uint32_t stage_tx = (uint32_t)(S * TC_TILE_BYTES + S * (BN * TC_BK * 2));   // bytes TMA brings per stage
    const size_t data_bytes = max((size_t)TC_STAGES * stage_bytes, (size_t)TC_STASH_BYTES);
    uint64_t* bars = (uint64_t*)(smem + data_bytes);
    uint64_t* full = bars;                 // [2]
    uint64_t* empty = bars + 2;            // [2]
    uint64_t* acc_full = bars + 4;
    uint64_t* acc_empty = bars + 5;
    uint32_t* tmem_holder = (uint32_t*)(bars + 6);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (p.Ncols + BN - 1) / BN;
    const int m0 = (blockIdx.x / n_tiles) * TC_BM;
    const int n0 = (blockIdx.x % n_tiles) * BN;
    // this CTA's K' range (split-K over blockIdx.y)
    const int kb0 = blockIdx.y * p.kps;
    const int nkb = min(p.nkb - kb0, p.kps);
    const int nchunks = (nkb + TC_CHUNK_KB - 1) / TC_CHUNK_KB;
    // first row of this product's blocks in the A and B maps (blocked products)
    const int rowA = p.zmode ? p.zA[blockIdx.z] * p.Ml : 0;
    const int rowB = p.zmode ? p.zB[blockIdx.z] * p.ml : 0;

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1); mbar_init(&full[1], 1);
        mbar_init(&empty[0], 1); mbar_init(&empty[1], 1);
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_holder))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *(volatile uint32_t*)tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA producer
            int kb_issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int st = kb & 1;
                const uint32_t use = (uint32_t)(kb >> 1);
                if (!mbar_wait(&empty[st], (use & 1u) ^ 1u, p.err)) break;
                unsigned char* base = smem + st * stage_bytes;
                mbar_expect_tx(&full[st], stage_tx);
                for (int s = 0; s < S; ++s)
                    tma_load_3d(base + s * TC_TILE_BYTES, &mapA, &full[st], (kb0 + kb) * TC_BK, m0 + rowA, s);
                for (int t = 0; t < S; ++t)
                    tma_load_3d(base + (S + t) * TC_TILE_BYTES, &mapB, &full[st], (kb0 + kb) * TC_BK, n0 + rowB, t);
                kb_issued = kb + 1;
            }
            // on an early exit, let the copies already issued land before the CTA ends
            if (kb_issued > 0 && kb_issued < nkb) {
                const int kb = kb_issued - 1;
                mbar_wait(&full[kb & 1], (uint32_t)((kb >> 1) & 1), p.err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = idesc_bf16_f32(TC_BM, BN);
            bool ok = true;
            for (int c = 0; c < nchunks && ok; ++c) {
                if (c > 0 && !mbar_wait(acc_empty, (uint32_t)((c - 1) & 1), p.err)) { ok = false; break; }
                tc_fence_after();
                const int kb_end = min(nkb, (c + 1) * TC_CHUNK_KB);
                for (int kb = c * TC_CHUNK_KB; kb < kb_end; ++kb) {
                    const int st = kb & 1;
                    if (!mbar_wait(&full[st], (uint32_t)((kb >> 1) & 1), p.err)) { ok = false; break; }
                    tc_fence_after();
                    // descriptors of slice tile 0 of A and of B in this stage; the start
                    // address field counts 16-byte units, so tile and K offsets add directly
                    const uint32_t base = smem_u32(smem + st * stage_bytes);
                    const uint64_t dA = sdesc_sw64(base), dB = sdesc_sw64(base + S * TC_TILE_BYTES);
                    const bool chunk_start = (kb == c * TC_CHUNK_KB);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
                        for (int s = 0; s < S; ++s) {
#pragma unroll
                            for (int t = 0; s + t < S; ++t) {
                                const int a = (s + t < TC_NACC - 1) ? s + t : TC_NACC - 1;
                                // the first MMA into each accumulator of a chunk overwrites it
                                const bool first = (kk == 0 && s == 0 && t < TC_NACC);
                                const uint32_t acc = (first && chunk_start) ? 0u : 1u;
                                umma_bf16(tmem + a * BN, dA + ((s * TC_TILE_BYTES + kk * 32) >> 4),
                                          dB + ((t * TC_TILE_BYTES + kk * 32) >> 4), idesc, acc);
                            }
                        }
                    }
                    umma_commit(&empty[st]);
                }
                if (ok) umma_commit(acc_full);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;       // column half: columns [64 half, min(BN, 64 half + 64))
        const int row = 32 * q + lane;
        float2* stash = reinterpret_cast<float2*>(smem);           // [128][BN + 1]
        // drains the accumulators chunk by chunk into (hi, lo) and stages them in the stash;
        // NCB 16-column blocks (compile time: 4, or (BN - 64) / 16 in the second half)
        auto drain = [&](auto ncb_c) -> bool {
            constexpr int NCB = decltype(ncb_c)::value;
            float hi[16 * NCB], lo[16 * NCB];
#pragma unroll
            for (int j = 0; j < 16 * NCB; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
            for (int c = 0; c < nchunks; ++c) {
                if (!mbar_wait(acc_full, (uint32_t)(c & 1), p.err)) return false;
                tc_fence_after();
                const int nacc = min(S, TC_NACC);   // accumulators the MMAs wrote (TMEM is not zeroed)
#pragma unroll
                for (int a = 0; a < TC_NACC; ++a) {
#pragma unroll
                    for (int cb = 0; cb < NCB; ++cb) {
                        float v[16];
                        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + a * BN + 64 * half + 16 * cb, v);
                        if (a < nacc) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) df_add(hi[16 * cb + j], lo[16 * cb + j], v[j]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
#pragma unroll
                for (int j = 0; j < 16 * NCB; ++j) {      // renormalise (hi, lo)
                    const float s = __fadd_rn(hi[j], lo[j]);
                    lo[j] = __fsub_rn(lo[j], __fsub_rn(s, hi[j]));
                    hi[j] = s;
                }
            }
            // stage (hi, lo) through the idle stage buffers (all TMA loads and MMAs are
            // done), then write out with a plain coalesced loop
#pragma unroll
            for (int j = 0; j < 16 * NCB; ++j) stash[row * (BN + 1) + 64 * half + j] = make_float2(hi[j], lo[j]);
            return true;
        };
        bool ok;
        if constexpr (BN == 128) ok = drain(std::integral_constant<int, 4>{});
        else ok = (half == 0) ? drain(std::integral_constant<int, 4>{}) : drain(std::integral_constant<int, (BN - 64) / 16>{});
        asm volatile("bar.sync 1, 256;" ::: "memory");          // the 8 epilogue warps
        if (ok && p.zmode) {
            // one real product: the tile's values, scaled by 2^(e_i + f_j - 14) of its blocks
            const int et = threadIdx.x - 64;
            const int z = blockIdx.z;
            const int* ea = p.ea + (int64_t)p.zA[z] * p.Ml;
            const int* eb = p.eb + (int64_t)p.zB[z] * p.ml;
            double* o = p.outr + (int64_t)(z * gridDim.y + blockIdx.y) * p.ml * p.Ml;
            const int nlr = min(TC_BM, p.Ml - m0), nlc = min(BN, p.ml - n0);
#pragma unroll 1
            for (int idx = et; idx < TC_BM * BN; idx += 256) {
                const int lr = idx % TC_BM, lc = idx / TC_BM;
                if (lr >= nlr || lc >= nlc) continue;
                const float2 v = stash[lr * (BN + 1) + lc];
                const int gi = m0 + lr, gj = n0 + lc;
                const long long sh = (long long)(ea[gi] + eb[gj] - 14) << 52;
                const long long b = __double_as_longlong(dfl_to(dfl{v.x, v.y}));
                o[(int64_t)gj * p.Ml + gi] = (b & 0x7FF0000000000000LL) ? __longlong_as_double(b + sh) : 0.0;
            }
        } else if (ok) {
            // combine the part products: complex A and B: re = RR - II, im = RI + IR; one
            // complex operand: its two part rows (or columns) are re and im
            const int et = threadIdx.x - 64;                       // 0..255
            const int rdiv = p.aC ? 2 : 1, cdiv = p.bC ? 2 : 1;
            const int NLR = TC_BM / rdiv, NLC = BN / cdiv;         // logical outputs per tile
            const int lr0 = m0 / rdiv, lc0 = n0 / cdiv;
            const int nlr = min(NLR, p.Ml - lr0), nlc = min(NLC, p.ml - lc0);
            auto V = [&](int rr, int cc) {
                const float2 v = stash[rr * (BN + 1) + cc];
                return dfl{v.x, v.y};
            };
            const bool plain = (p.alpha == 1.0 && p.beta == 0.0);
#pragma unroll 1
            for (int idx = et; idx < NLR * NLC; idx += 256) {
                int lr, lc;
                if (p.transposed) { lc = idx % NLC; lr = idx / NLC; }
                else { lr = idx % NLR; lc = idx / NLR; }
                if (lr >= nlr || lc >= nlc) continue;
                const int gi = lr0 + lr, gj = lc0 + lc;
                dfl dre, dim;
                if (p.aC && p.bC) {
                    dre = dfl_sub(V(2 * lr, 2 * lc), V(2 * lr + 1, 2 * lc + 1));
                    dim = dfl_add(V(2 * lr, 2 * lc + 1), V(2 * lr + 1, 2 * lc));
                } else if (p.aC) {
                    dre = V(2 * lr, lc);
                    dim = V(2 * lr + 1, lc);
                } else {
                    dre = V(lr, 2 * lc);
                    dim = V(lr, 2 * lc + 1);
                }
                // times 2^(e_i + f_j - 14), exactly, on the exponent fields (normal values)
                const long long sh = (long long)(p.ea[gi] + p.eb[gj] - 14) << 52;
                const double r0 = dfl_to(dre), i0 = dfl_to(dim);
                const long long br = __double_as_longlong(r0), bi = __double_as_longlong(i0);
                const double re = (br & 0x7FF0000000000000LL) ? __longlong_as_double(br + sh) : 0.0;
                const double im = (bi & 0x7FF0000000000000LL) ? __longlong_as_double(bi + sh) : 0.0;
                if (p.part) {
                    p.part[((int64_t)blockIdx.y * p.ml + gj) * p.Ml + gi] = make_double2(re, im);
                    continue;
                }
                double2* o = p.transposed ? (p.out + (int64_t)gj + (int64_t)gi * p.ldo)
                                          : (p.out + (int64_t)gi + (int64_t)gj * p.ldo);
                if (plain) { *o = make_double2(re, im); continue; }
                double2 val = make_double2(p.alpha * re, p.alpha * im);
                if (p.beta != 0.0) {
                    const double2 old = *o;
                    val.x += p.beta * old.x;
                    val.y += p.beta * old.y;
                }
                *o = val;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// ------------------------------------------------------------------------------ slicing
// Row exponents of A'.  A_op[i, k] = src[i*sa_i + k*sa_k] (complex); e_i = frexp exponent
// of max_k max(|Re|, |Im|) so that |x| 2^-e_i < 1.
// band >= 0 (square operators): entries with cyclic |i - k| <= band are excluded (they are
// applied separately in FP64).
__device__ __forceinline__ bool in_band(int64_t i, int64_t k, int64_t K, int band) {
    if (band < 0) return false;
    int64_t d = i - k;
    if (d < 0) d = -d;
    if (K - d < d) d = K - d;
    return d <= band;
}

// Exponents are taken from the IEEE exponent fields with integer operations (GB300's FP64
// pipe is 1/64 of its FP32 rate): for a normal double with biased exponent E, frexp gives
// E - 1022, and the largest magnitude of a row carries its largest exponent field.
__device__ __forceinline__ int exp_field(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

__global__ void k_exp_rows(const void* src, int is_real, int64_t M, int64_t K, int64_t sa_i, int64_t sa_k, int band,
                           int* e) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (i >= M) return;
    int mx = 0;
    for (int64_t k = threadIdx.x & 31; k < K; k += 32) {
        if (in_band(i, k, K, band)) continue;
        if (is_real) {
            mx = max(mx, exp_field(((const double*)src)[i * sa_i + k * sa_k]));
        } else {
            const double2 v = ((const double2*)src)[i * sa_i + k * sa_k];
            mx = max(mx, max(exp_field(v.x), exp_field(v.y)));
        }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) e[i] = mx ? mx - 1022 : 0;
}

// Row exponents from the exponent fields gathered during the assembly (the values
// k_exp_rows gives for those entries)
__global__ void k_exp_from_fields(const int* fields, int64_t M, int* e) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int mx = fields[i];
    e[i] = mx ? mx - 1022 : 0;
}

// B column exponents: B_op[k, j] = src[k*sb_k + j*sb_j] (complex, or real when is_real);
// f_j scales both part rows of column j.  One CTA per column, four loads in flight per thread.
__global__ void __launch_bounds__(256) k_exp_cols(const void* src, int is_real, int64_t K, int64_t m, int64_t sb_k,
                                                  int64_t sb_j, int* f) {
    __shared__ int red[8];
    const int64_t j = blockIdx.x;
    int mx = 0;
    for (int64_t k0 = threadIdx.x; k0 < K; k0 += 4 * (int64_t)blockDim.x) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + (int64_t)u * blockDim.x;
            if (k >= K) break;
            if (is_real) {
                mx = max(mx, exp_field(((const double*)src)[k * sb_k + j * sb_j]));
            } else {
                const double2 v = ((const double2*)src)[k * sb_k + j * sb_j];
                mx = max(mx, max(exp_field(v.x), exp_field(v.y)));
            }
        }
    }
    mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mx = max(mx, red[q]);
        f[j] = mx ? mx - 1022 : 0;
    }
}

// float bits of d 2^{-7s} for an integer |d| <= 128, whose upper half is the bf16 value
// (at most 8 significant bits): adding d to the bit pattern of C = 1.5 2^{23-7s}, whose
// ulp is 2^{-7s}, gives C + d 2^{-7s} exactly, and subtracting C leaves d 2^{-7s} (one
// integer add and one FADD; checked against the scaled conversion for every d and s)
__device__ __forceinline__ uint32_t digit_bits(int d, int s) {
    const float c = __int_as_float((127 + 23 - 7 * s) << 23) * 1.5f;   // a constant per unrolled s
    return __float_as_uint(__fsub_rn(__int_as_float(__float_as_int(c) + d), c));
}

// val 2^-e in (-1, 1) -> S slices: X = round(val 2^{7S - e}) (one rounding, half away from
// zero), then balanced base-128 digits from the least significant up: d in [-64, 63] for
// s >= 1 and the leading |d_0| <= 128; slice s stores d_s 2^{-7s} (exact in bf16), returned
// here as float bit patterns whose upper halves are the bf16 values.  X is formed from the significand and exponent fields with
// integer shifts: |val| < 2^e makes the right shift 1075 + e - 7S - E at least 53 - 7S > 0.
// Zeros and subnormals give 0.
__device__ __forceinline__ void split_digits(double val, int e, int S, uint32_t* d) {
    const long long b = __double_as_longlong(val);
    const int E = (int)((b >> 52) & 0x7FF);
    const int sh = 1075 + e - 7 * S - E;
    long long X = 0;
    if (E != 0 && sh < 63) {
        const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        X = (m + (1LL << (sh - 1))) >> sh;
        if (b < 0) X = -X;
    }
    if (S >= 4) {
        // |X| < 2^(7S) <= 2^49: the three lowest digits come from the low 21 bits and the rest
        // from the upper part plus the carry, all in 32-bit integers
        int cur = (int)(X & 0x1FFFFF);
        const int hi = (int)(X >> 21);
        int t = 0;
#pragma unroll
        for (int s = TC_SMAX - 1; s >= 1; --s) {
            if (s >= S) { d[s] = 0u; continue; }
            if (t == 3) cur += hi;
            int q = cur & 127;
            if (q >= 64) q -= 128;
            cur = (cur - q) >> 7;
            d[s] = digit_bits(q, s);
            ++t;
        }
        if (t == 3) cur += hi;                  // S = 4: the upper part is the leading digit
        d[0] = digit_bits(cur, 0);
        return;
    }
#pragma unroll
    for (int s = TC_SMAX - 1; s >= 1; --s) {
        if (s >= S) { d[s] = 0u; continue; }
        int q = (int)(X & 127);
        if (q >= 64) q -= 128;
        X = (X - q) >> 7;
        d[s] = digit_bits(q, s);
    }
    d[0] = digit_bits((int)X, 0);
}

// Planar slices.  A operand (M x K): a complex row i becomes rows 2i (real part) and 2i+1
// (imaginary part, negated when conj), a real row i stays row i; B operand (K x m) likewise
// by columns (stored K-major: out[s][row][k]).  The product of the part matrices gives the
// four (or two) real products the epilogue combines, so a real operand costs half of a
// complex one.  Each thread takes SLICE_VEC consecutive k (Kp is a multiple of 32, so a
// group never straddles a row) and writes 16 bytes per part row and slice.
#define SLICE_VEC 8
// digits of SLICE_VEC values (one part row) packed as bf16 pairs, then one 16-byte store per slice
// The same digits with the slice count SC known at compile time: below the leading digit,
// the balanced digits of X are the plain base-128 digits of X + 64 (1 + 128 + ... +
// 128^(SC-2)), less 64 each, and the leading digit is what lies above them (an arithmetic
// shift), so every digit is one shift, one mask and one subtraction of the biased integer
// (equal digit for digit to the carry loop above, for every |X| <= 2^(7 SC)).
template <int SC>
__device__ __forceinline__ void split_digits_c(double val, int e, uint32_t* d) {
    const long long b = __double_as_longlong(val);
    const int E = (int)((b >> 52) & 0x7FF);
    const int sh = 1075 + e - 7 * SC - E;
    long long X = 0;
    if (E != 0 && sh < 63) {
        const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        X = (m + (1LL << (sh - 1))) >> sh;
        if (b < 0) X = -X;
    }
    constexpr long long C = 64LL * ((1LL << (7 * (SC - 1))) - 1) / 127;
    const long long Y = X + C;
    d[0] = digit_bits((int)(Y >> (7 * (SC - 1))), 0);
#pragma unroll
    for (int s = 1; s < SC; ++s) d[s] = digit_bits((int)((Y >> (7 * (SC - 1 - s))) & 127) - 64, s);
#pragma unroll
    for (int s = SC; s < TC_SMAX; ++s) d[s] = 0u;
}

// SC > 0: the slice count is SC (compile time; S is ignored); SC = 0: S at run time
template <int SC = 0, class Get>
__device__ __forceinline__ void slice_part(Get v, int e, int S, __nv_bfloat16* out, int64_t row, int64_t Kp,
                                           int64_t k0, size_t stride) {
    if (SC > 0) S = SC;
    uint32_t w[TC_SMAX][SLICE_VEC / 2];
    uint32_t ev[TC_SMAX];
#pragma unroll
    for (int u = 0; u < SLICE_VEC; ++u) {
        uint32_t d[TC_SMAX];
        if constexpr (SC > 0) split_digits_c<SC>(v(u), e, d);
        else split_digits(v(u), e, S, d);
        // two values' bf16 halves into one word: the even value low, the odd one high
#pragma unroll
        for (int s = 0; s < TC_SMAX; ++s) {
            if ((u & 1) == 0) ev[s] = d[s];
            else w[s][u >> 1] = __byte_perm(ev[s], d[s], 0x7632);
        }
    }
    uint4* o = reinterpret_cast<uint4*>(out + row * Kp + k0);
    const size_t st16 = stride / 8;                // one slice, in 16-byte units
#pragma unroll
    for (int s = 0; s < TC_SMAX; ++s)
        if (s < S) o[s * st16] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// Contiguous complex rows (unit stride along k): the warp reads its 32 * SLICE_VEC values
// coalesced (one 512-byte run per load) into shared memory, then each lane takes SLICE_VEC
// consecutive values.  One pad slot per 8 keeps both phases free of bank conflicts.
// BLOCKS 0: part rows 2i (Re) and 2i+1 (Im); BLOCKS 3: row blocks [Re; Im; Re + Im] of M
// rows each, block b of row i scaled by e[b M + i], the sum block with its leading S3 <= S
// slices only (the products that use it take no more; the rest of its slices stay unwritten)
// SC, SC3 > 0: the slice counts S and S3 at compile time (the common ones), 0: at run time
template <int BLOCKS, int SC, int SC3>
__global__ void __launch_bounds__(256, BLOCKS ? 3 : 4) k_slice_A_rows(const double2* src, int conj, int64_t M, int64_t K,
                                                                    int64_t Kp, int64_t sa_i, int band, const int* e,
                                                                    int S, __nv_bfloat16* out, int S3) {
    constexpr int blocks = BLOCKS;
    const int64_t i = blockIdx.y;
    __shared__ double2 stage[8][32 * SLICE_VEC + 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t kw = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * SLICE_VEC;
    const double2* rowp = src + i * sa_i;
#pragma unroll
    for (int u = 0; u < SLICE_VEC; ++u) {
        const int q = u * 32 + lane;
        const int64_t k = kw + q;
        double2 x = make_double2(0.0, 0.0);
        if (k < K && !in_band(i, k, K, band)) x = rowp[k];
        stage[w][q + (q >> 3)] = x;
    }
    __syncwarp();
    const int64_t k0 = kw + lane * SLICE_VEC;
    if (k0 >= Kp) return;
    const size_t stride = (size_t)((blocks ? blocks : 2) * M) * Kp;
    // real parts, then imaginary parts (then their sums), each value read from shared
    // memory when it is split
    const double2* st = stage[w];
    const int64_t rre = blocks ? i : 2 * i, rim = blocks ? M + i : 2 * i + 1;
    slice_part<SC>([&](int u) { const int q = lane * SLICE_VEC + u; return st[q + (q >> 3)].x; }, e[i], S, out,
               rre, Kp, k0, stride);
    slice_part<SC>([&](int u) { const int q = lane * SLICE_VEC + u; const double y = st[q + (q >> 3)].y; return conj ? -y : y; },
               e[blocks ? M + i : i], S, out, rim, Kp, k0, stride);
    if (BLOCKS == 3)
        slice_part<SC3>([&](int u) {
                       const int q = lane * SLICE_VEC + u;
                       const double2 x = st[q + (q >> 3)];
                       return x.x + (conj ? -x.y : x.y);
                   },
                   e[2 * M + i], S3, out, 2 * M + i, Kp, k0, stride);
}

__global__ void k_slice_A(const void* src, int is_real, int conj, int64_t M, int64_t K, int64_t Kp, int64_t sa_i,
                          int64_t sa_k, int band, const int* e, int S, __nv_bfloat16* out) {
    const int64_t i = blockIdx.y;
    const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * SLICE_VEC;
    if (k0 >= Kp || i >= M) return;
    const int ei = e[i];
    double re[SLICE_VEC], im[SLICE_VEC];
#pragma unroll
    for (int u = 0; u < SLICE_VEC; ++u) {
        const int64_t k = k0 + u;
        re[u] = 0.0; im[u] = 0.0;
        if (k < K && !in_band(i, k, K, band)) {
            if (is_real) {
                re[u] = ((const double*)src)[i * sa_i + k * sa_k];
            } else {
                const double2 x = ((const double2*)src)[i * sa_i + k * sa_k];
                re[u] = x.x; im[u] = conj ? -x.y : x.y;
            }
        }
    }
    const int64_t rows = is_real ? M : 2 * M;
    const size_t stride = (size_t)rows * Kp;
    slice_part([&](int u) { return re[u]; }, ei, S, out, is_real ? i : 2 * i, Kp, k0, stride);
    if (!is_real) slice_part([&](int u) { return im[u]; }, ei, S, out, 2 * i + 1, Kp, k0, stride);
}

// blocks as in k_slice_A_rows, by columns (complex B only)
__global__ void k_slice_B(const void* src, int is_real, int64_t K, int64_t m, int64_t Kp, int64_t sb_k,
                          int64_t sb_j, const int* f, int S, __nv_bfloat16* out, int blocks) {
    const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * SLICE_VEC;
    const int64_t j = blockIdx.y;
    if (k0 >= Kp || j >= m) return;
    const int fe = f[j];
    double re[SLICE_VEC], im[SLICE_VEC];
#pragma unroll
    for (int u = 0; u < SLICE_VEC; ++u) {
        const int64_t k = k0 + u;
        re[u] = 0.0; im[u] = 0.0;
        if (k < K) {
            if (is_real) { re[u] = ((const double*)src)[k * sb_k + j * sb_j]; }
            else { const double2 x = ((const double2*)src)[k * sb_k + j * sb_j]; re[u] = x.x; im[u] = x.y; }
        }
    }
    if (blocks) {
        const size_t stride = (size_t)(blocks * m) * Kp;
        slice_part([&](int u) { return re[u]; }, fe, S, out, j, Kp, k0, stride);
        slice_part([&](int u) { return im[u]; }, f[m + j], S, out, m + j, Kp, k0, stride);
        if (blocks == 3) slice_part([&](int u) { return re[u] + im[u]; }, f[2 * m + j], S, out, 2 * m + j, Kp, k0, stride);
        return;
    }
    const int64_t rows = is_real ? m : 2 * m;
    const size_t stride = (size_t)rows * Kp;
    slice_part([&](int u) { return re[u]; }, fe, S, out, is_real ? j : 2 * j, Kp, k0, stride);
    if (!is_real) slice_part([&](int u) { return im[u]; }, fe, S, out, 2 * j + 1, Kp, k0, stride);
}

// exponents of the row blocks from those of the complex rows (e[0..M)): the Re and Im
// blocks keep e_i (max(|Re|, |Im|) < 2^e_i), the sum block takes e_i + 1 (|Re + Im| < 2^(e_i + 1))
__global__ void k_exp_blocks(int* e, int64_t M, int blocks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int v = e[i];
    e[M + i] = v;
    if (blocks == 3) e[2 * M + i] = v + 1;
}

// ------------------------------------------------------------------------------ host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static PFN_encodeTiled g_encode = nullptr;
static std::mutex g_encode_mutex;

static bem_status get_encode(bem_ctx* h) {
    std::lock_guard<std::mutex> lk(g_encode_mutex);
    if (g_encode) return BEM_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess)
        return bem_fail(h, BEM_E_CUDA, "cuTensorMapEncodeTiled is not available");
    g_encode = (PFN_encodeTiled)fn;
    return BEM_OK;
}

struct TcOperand {
    __nv_bfloat16* slices = nullptr;  // S x rows x Kp
    int* exps = nullptr;              // rows
    int64_t rows = 0, Kp = 0, K = 0;
    size_t cap = 0;                   // bytes allocated for slices
    size_t exp_cap = 0;
    int cplx = 1;                     // complex operand: real and imaginary parts in separate rows
    int64_t lrows = 0;                // logical rows (A) / columns (B): rows = (cplx ? 2 : 1) lrows
    int nslices = 0;                  // slices the map spans
    int blocks = 0;                   // 0: part rows (above); 2, 3: real row blocks of lrows rows
                                      // each (Re, Im, and Re + Im for 3), cplx = 0
    int s3 = 0;                       // slices the Re + Im block holds (A operands)
    CUtensorMap map;
};

// The real products of blocked operands that make one complex product: product z
// multiplies row block zA[z] of A by row block zB[z] of B; gauss = 1 combines three as
// C = (P0 - P1) + i (P2 - P0 - P1) (Gauss's three-multiplication form, A and B blocked
// [Re; Im; Re + Im]), gauss = 0 two as C = P0 + i P1 (A blocked [Re; Im], B real).
struct TcBlocks {
    int nz;
    int zA[3], zB[3];
    int gauss;
};

struct TcState {
    int S = 6;                        // slices per operand (3..TC_SMAX), 6 = 42 bits
    TcOperand opS, opW, opD;          // A operands: X^T of the assembled matrices
    TcOperand opVh, opU;              // Woodbury factors
    TcOperand bbuf;                   // B operand scratch (reused)
    TcOperand bbuf_rhs;               // the right-hand sides' B operand while they run on the
                                      // auxiliary stream (bem_factor_rhs_planewave)
    TcOperand tmpA;                   // A operand scratch (reused)
    double2* part = nullptr;          // split-K partials
    size_t part_cap = 0;
    double* zbuf = nullptr;           // real products of the blocked path
    size_t zbuf_cap = 0;
};

static TcState* tcs(bem_ctx* h) {
    if (!h->tc) {
        TcState* t = new TcState();
        if (h->opt.split_slices >= 3 && h->opt.split_slices <= TC_SMAX) t->S = h->opt.split_slices;
        h->tc = t;
    }
    return (TcState*)h->tc;
}

static int64_t pad32(int64_t x) { return (x + 31) / 32 * 32; }   // K, padded to whole 32-wide K blocks

// tensor map of an operand's slices: boxes of TC_BK (K') x box_rows (rows) x 1 (slice)
static bem_status encode_map_box(bem_ctx* h, const TcOperand& op, int S, int box_rows, CUtensorMap* map) {
    bem_status st = get_encode(h);
    if (st != BEM_OK) return st;
    cuuint64_t dims[3] = {(cuuint64_t)op.Kp, (cuuint64_t)op.rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)(op.Kp * 2), (cuuint64_t)(op.Kp * op.rows * 2)};
    cuuint32_t box[3] = {TC_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op.slices, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return bem_fail(h, BEM_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return BEM_OK;
}
static bem_status encode_map(bem_ctx* h, TcOperand& op, int S) {
    op.nslices = S;
    return encode_map_box(h, op, S, TC_BM, &op.map);
}

static bem_status reserve(bem_ctx* h, TcOperand& op, int64_t rows, int64_t Kp, int S) {
    const size_t need = (size_t)S * rows * Kp * sizeof(__nv_bfloat16);
    if (need > op.cap) {
        if (op.slices) { cudaStreamSynchronize(h->stream); bem_dfree(h, op.slices); op.slices = nullptr; op.cap = 0; }
        BEM_CUDA(h, bem_dmalloc(h, (void**)&op.slices, need));
        op.cap = need;
    }
    if ((size_t)rows * sizeof(int) > op.exp_cap) {
        if (op.exps) { cudaStreamSynchronize(h->stream); bem_dfree(h, op.exps); op.exps = nullptr; op.exp_cap = 0; }
        BEM_CUDA(h, bem_dmalloc(h, (void**)&op.exps, (size_t)rows * sizeof(int)));
        op.exp_cap = (size_t)rows * sizeof(int);
    }
    op.rows = rows;
    op.Kp = Kp;
    return BEM_OK;
}

// A operand: rows M, K complex columns, A_op[i,k] = src[i*sa_i + k*sa_k]; band >= 0 drops
// the cyclic band |i - k| <= band (square operators)
// k_slice_A_rows with the slice counts of the defaults (6 per operand, 5 for the
// right-hand-side product) compiled in, any other at run time
static void launch_slice_rows(int blocks, const double2* src, int conj, int64_t M, int64_t K, int64_t Kp, int64_t sa_i,
                              int band, const int* e, int S, __nv_bfloat16* out, int S3, dim3 grid, cudaStream_t st) {
    if (blocks) {
        if (S == 6 && S3 == 5) k_slice_A_rows<3, 6, 5><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, S3);
        else if (S == 6 && S3 == 6) k_slice_A_rows<3, 6, 6><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, S3);
        else if (S == 5 && S3 == 5) k_slice_A_rows<3, 5, 5><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, S3);
        else k_slice_A_rows<3, 0, 0><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, S3);
    } else {
        if (S == 6) k_slice_A_rows<0, 6, 0><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, 0);
        else if (S == 5) k_slice_A_rows<0, 5, 0><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, 0);
        else k_slice_A_rows<0, 0, 0><<<grid, 256, 0, st>>>(src, conj, M, K, Kp, sa_i, band, e, S, out, 0);
    }
}

// blocks 2 or 3: real row blocks [Re; Im] or [Re; Im; Re + Im] (complex rows with unit
// stride along k only)
static bem_status slice_A(bem_ctx* h, TcOperand& op, const void* src, int64_t M, int64_t K, int64_t sa_i, int64_t sa_k,
                          int band = -1, int is_real = 0, int conj = 0, const int* fields = nullptr, int blocks = 0,
                          int S3 = 0) {
    const int S = tcs(h)->S;
    const int64_t Kp = pad32(K);
    if (blocks && (is_real || sa_k != 1 || blocks != 3 || S3 < 1 || S3 > S))
        return bem_fail(h, BEM_E_INVALID, "slice_A: row blocks need complex rows with unit stride");
    bem_status st = reserve(h, op, blocks ? blocks * M : (is_real ? M : 2 * M), Kp, S);
    if (st != BEM_OK) return st;
    op.K = K;
    op.cplx = (is_real || blocks) ? 0 : 1;
    op.blocks = blocks;
    op.s3 = blocks == 3 ? S3 : S;
    op.lrows = M;
    if (fields) {
        BEM_TIMED(h, "k_exp_rows", (k_exp_from_fields<<<(unsigned)((M + 255) / 256), 256, 0, h->stream>>>(fields, M, op.exps)));
    } else {
        BEM_TIMED(h, "k_exp_rows", (k_exp_rows<<<(unsigned)((M + 7) / 8), 256, 0, h->stream>>>(src, is_real, M, K, sa_i, sa_k, band, op.exps)));
    }
    BEM_LAUNCH(h, "k_exp_rows");
    if (blocks) {
        BEM_TIMED(h, "k_exp_rows", (k_exp_blocks<<<(unsigned)((M + 255) / 256), 256, 0, h->stream>>>(op.exps, M, blocks)));
        BEM_LAUNCH(h, "k_exp_blocks");
    }
    dim3 grid((unsigned)((Kp / SLICE_VEC + 255) / 256), (unsigned)M);
    if (blocks || (!is_real && sa_k == 1))
        BEM_TIMED(h, "k_slice_A", (launch_slice_rows(blocks, (const double2*)src, conj, M, K, Kp, sa_i, band, op.exps, S,
                                                     op.slices, S3, grid, h->stream)));
    else
        BEM_TIMED(h, "k_slice_A", (k_slice_A<<<grid, 256, 0, h->stream>>>(src, is_real, conj, M, K, Kp, sa_i, sa_k, band, op.exps, S, op.slices)));
    BEM_LAUNCH(h, "k_slice_A");
    return encode_map(h, op, S);
}

// B operand: K x m (complex or real), B_op[k,j] = src[k*sb_k + j*sb_j]
// (blocks 2 or 3: real row blocks of the columns, as in slice_A; complex B only)
static bem_status slice_B(bem_ctx* h, TcOperand& op, const void* src, int is_real, int64_t K, int64_t m, int64_t sb_k,
                          int64_t sb_j, int S_over = 0, int blocks = 0) {
    const int S = S_over ? S_over : tcs(h)->S;
    const int64_t Kp = pad32(K);
    if (blocks && (is_real || blocks < 2 || blocks > 3))
        return bem_fail(h, BEM_E_INVALID, "slice_B: row blocks need a complex operand");
    bem_status st = reserve(h, op, blocks ? blocks * m : (is_real ? m : 2 * m), Kp, S);
    if (st != BEM_OK) return st;
    op.K = K;
    op.cplx = (is_real || blocks) ? 0 : 1;
    op.blocks = blocks;
    op.s3 = S;
    op.lrows = m;
    BEM_TIMED(h, "k_exp_cols", (k_exp_cols<<<(unsigned)m, 256, 0, h->stream>>>(src, is_real, K, m, sb_k, sb_j, op.exps)));
    BEM_LAUNCH(h, "k_exp_cols");
    if (blocks) {
        BEM_TIMED(h, "k_exp_cols", (k_exp_blocks<<<(unsigned)((m + 255) / 256), 256, 0, h->stream>>>(op.exps, m, blocks)));
        BEM_LAUNCH(h, "k_exp_blocks");
    }
    dim3 grid((unsigned)((Kp / SLICE_VEC + 255) / 256), (unsigned)m);
    // contiguous complex columns have the layout of contiguous A rows: the row slicer's
    // coalesced staging serves them (column j as row j, no band, no conjugation)
    if (!is_real && sb_k == 1)
        BEM_TIMED(h, "k_slice_B", (launch_slice_rows(blocks, (const double2*)src, 0, m, K, Kp, sb_j, -1, op.exps, S,
                                                     op.slices, S, grid, h->stream)));
    else
        BEM_TIMED(h, "k_slice_B", (k_slice_B<<<grid, 256, 0, h->stream>>>(src, is_real, K, m, Kp, sb_k, sb_j, op.exps, S, op.slices, blocks)));
    BEM_LAUNCH(h, "k_slice_B");
    return encode_map(h, op, S);
}

static size_t gemm_smem(int S) {
    const size_t data = std::max((size_t)TC_STAGES * 2 * S * TC_TILE_BYTES, (size_t)TC_STASH_BYTES);
    return data + 64 + 1024;    // barriers + TMEM address, and slack for 1024-byte alignment
}

// out = alpha (A B) + beta out for sliced operands (complex result, M x m)
// out = alpha sum_s part[s] + beta out over the M x m split partials
__global__ void k_splitk_reduce(const double2* __restrict__ part, int splits, int M, int m, double2* out, int64_t ldo,
                                int transposed, double alpha, double beta) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * m) return;
    const int i = (int)(idx % M), j = (int)(idx / M);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
        const double2 v = part[(int64_t)s * M * m + idx];
        re += v.x;
        im += v.y;
    }
    double2* o = transposed ? (out + (int64_t)j + (int64_t)i * ldo) : (out + (int64_t)i + (int64_t)j * ldo);
    double2 val = make_double2(alpha * re, alpha * im);
    if (beta != 0.0) {
        const double2 old = *o;
        val.x += beta * old.x;
        val.y += beta * old.y;
    }
    *o = val;
}

// out = alpha C + beta out from the real products of blocked operands (TcBlocks), summed
// over the K' splits: P[(z splits + s) M m + j M + i].  32 x 32 tiles of (i, j) per CTA of
// 32 x 8 threads: the products are read along i; a transposed output (out[j + i ldo]) is
// staged through shared memory so that it is written along j.
__global__ void __launch_bounds__(256) k_combine_blocks(const double* __restrict__ P, int splits, int gauss, int M, int m,
                                                        double2* out, int64_t ldo, int transposed, double alpha,
                                                        double beta) {
    __shared__ double2 tile[32][33];
    const int64_t plane = (int64_t)M * m;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nz = gauss ? 3 : 2;
    auto value = [&](int i, int j) {
        double pz[3] = {0.0, 0.0, 0.0};
        const int64_t idx = (int64_t)j * M + i;
        for (int z = 0; z < nz; ++z)
            for (int s = 0; s < splits; ++s) pz[z] += P[(int64_t)(z * splits + s) * plane + idx];
        const double re = gauss ? pz[0] - pz[1] : pz[0];
        const double im = gauss ? (pz[2] - pz[0]) - pz[1] : pz[1];
        return make_double2(alpha * re, alpha * im);
    };
    auto store = [&](double2* o, double2 val) {
        if (beta != 0.0) {
            const double2 old = *o;
            val.x += beta * old.x;
            val.y += beta * old.y;
        }
        *o = val;
    };
    if (!transposed) {
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + tx, j = j0 + r;
            if (i < M && j < m) store(out + (int64_t)i + (int64_t)j * ldo, value(i, j));
        }
        return;
    }
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + tx, j = j0 + r;
        if (i < M && j < m) tile[r][tx] = value(i, j);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + tx;
        if (i < M && j < m) store(out + (int64_t)j + (int64_t)i * ldo, tile[tx][r]);
    }
}

// The same for an output stored in the products' own order (out[i + j ldo]): a flat grid,
// two consecutive entries per thread, every plane's loads issued before they are combined
// (the splits summed in the same order as above).
__global__ void __launch_bounds__(256) k_combine_blocks_flat(const double* __restrict__ P, int splits, int gauss,
                                                             int M, int m, double2* out, int64_t ldo, double alpha,
                                                             double beta) {
    const int64_t plane = (int64_t)M * m;
    const int64_t base = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (base >= plane) return;
    const bool two = base + 1 < plane;
    const int nz = gauss ? 3 : 2;
    double v0[3] = {0.0, 0.0, 0.0}, v1[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < splits; ++s) {
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            if (z >= nz) break;
            const double* q = P + (int64_t)(z * splits + s) * plane + base;
            v0[z] += __ldcs(q);
            if (two) v1[z] += __ldcs(q + 1);
        }
    }
    for (int u = 0; u < (two ? 2 : 1); ++u) {
        const double* v = u ? v1 : v0;
        const double re = gauss ? v[0] - v[1] : v[0];
        const double im = gauss ? (v[2] - v[0]) - v[1] : v[1];
        const int64_t e = base + u;
        int64_t i, j;
        if (plane < (1LL << 32)) {                      // 32-bit division where it suffices
            i = (unsigned)e % (unsigned)M;
            j = (unsigned)e / (unsigned)M;
        } else {
            i = e % M;
            j = e / M;
        }
        double2* o = out + i + j * ldo;
        double2 val = make_double2(alpha * re, alpha * im);
        if (beta != 0.0) {
            const double2 old = *o;
            val.x += beta * old.x;
            val.y += beta * old.y;
        }
        *o = val;
    }
}

// S_use > 0: multiply with the leading S_use digit slices only (B sliced with S_use, A with
// at least that many).  zb: the complex product as real products of blocked operands
// (A.blocks > every zA, B blocked likewise or real).
static bem_status tc_gemm(bem_ctx* h, const TcOperand& A, const TcOperand& B, cplx* out, int64_t ldo, int transposed,
                          double alpha, double beta, const char* tag, int S_use = 0, const TcBlocks* zb = nullptr) {
    TcState* t = tcs(h);
    if (A.Kp != B.Kp) return bem_fail(h, BEM_E_INVALID, "tc_gemm: K mismatch");
    const int Sg = S_use ? S_use : t->S;
    if (Sg > t->S) return bem_fail(h, BEM_E_INVALID, "tc_gemm: more slices than the operands hold");
    TcGemmArgs p;
    p.M = (int)A.rows;
    p.Ncols = (int)B.rows;
    p.Ml = (int)A.lrows;
    p.ml = (int)B.lrows;
    p.aC = A.cplx;
    p.bC = B.cplx;
    p.zmode = 0;
    p.outr = nullptr;
    const int nz = zb ? zb->nz : 1;
    if (zb) {
        if (zb->nz != (zb->gauss ? 3 : 2)) return bem_fail(h, BEM_E_INVALID, "tc_gemm: blocked product count");
        for (int z = 0; z < nz; ++z) {
            const int bb = B.blocks ? B.blocks : (B.cplx ? 0 : 1);
            if (zb->zA[z] < 0 || zb->zA[z] >= A.blocks || zb->zB[z] < 0 || zb->zB[z] >= bb)
                return bem_fail(h, BEM_E_INVALID, "tc_gemm: operand blocks do not match the products");
            if ((zb->zA[z] == 2 && Sg > A.s3) || (zb->zB[z] == 2 && Sg > B.s3))
                return bem_fail(h, BEM_E_INVALID, "tc_gemm: the sum block holds fewer slices");
            p.zA[z] = zb->zA[z];
            p.zB[z] = zb->zB[z];
        }
        p.zmode = 1;
        p.M = p.Ml;
        p.Ncols = p.ml;
    } else {
        if (A.blocks || B.blocks) return bem_fail(h, BEM_E_INVALID, "tc_gemm: blocked operands need their products");
        if (!A.cplx && !B.cplx) return bem_fail(h, BEM_E_INVALID, "tc_gemm: at least one operand must be complex");
    }
    p.nkb = (int)(A.Kp / TC_BK);
    p.S = Sg;
    p.ea = A.exps;
    p.eb = B.exps;
    p.out = out;
    p.ldo = ldo;
    p.transposed = transposed;
    p.alpha = alpha;
    p.beta = beta;
    p.err = h->dev_err;
    p.kps = p.nkb;
    p.part = nullptr;
    const size_t smem = gemm_smem(Sg);
    // the stage's tile choice (bem_options): the filter products, the right-hand-side product,
    // or automatic for the others
    const bool is_filter = strncmp(tag, "tc_filter", 9) == 0, is_rhs = strcmp(tag, "tc_rhs_SY") == 0;
    const int want_bn = is_filter ? h->opt.filter_tile_n : (is_rhs ? h->opt.rhs_tile_n : 0);
    const int want_split = is_filter ? h->opt.filter_split_k : (is_rhs ? h->opt.rhs_split_k : 0);
    // tile width: 112 when it pads the B part rows less than 128 does (the filter's 201 real
    // or 2 x 201 complex columns: 224 and 448 instead of 256 and 512), for the usual slice counts
    const int pad128 = (p.Ncols + 127) / 128 * 128, pad112 = (p.Ncols + 111) / 112 * 112;
    int BN = (pad112 < pad128 && (Sg == 5 || Sg == 6)) ? 112 : 128;
    if (want_bn == 128 || (want_bn == 112 && (Sg == 5 || Sg == 6))) BN = want_bn;
    void (*kern)(const CUtensorMap, const CUtensorMap, TcGemmArgs) = nullptr;
    switch (Sg * 1000 + BN) {
        case 3128: kern = k_tc_gemm<3, 128>; break;
        case 4128: kern = k_tc_gemm<4, 128>; break;
        case 5128: kern = k_tc_gemm<5, 128>; break;
        case 6128: kern = k_tc_gemm<6, 128>; break;
        case 7128: kern = k_tc_gemm<7, 128>; break;
        case 5112: kern = k_tc_gemm<5, 112>; break;
        case 6112: kern = k_tc_gemm<6, 112>; break;
        default: return bem_fail(h, BEM_E_UNSUPPORTED, "tc_gemm: slices per operand must be 3..7");
    }
    CUtensorMap mapB = B.map;
    if (BN != TC_BM) {
        bem_status st = encode_map_box(h, B, B.nslices, BN, &mapB);
        if (st != BEM_OK) return st;
    }
    BEM_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int mt = (p.M + TC_BM - 1) / TC_BM, nt = (p.Ncols + BN - 1) / BN;
    // split K' across CTAs (FP64 partials summed by k_splitk_reduce) when that fills the
    // SMs better: every tile costs the same, so the run time is (waves of CTAs) x (chunks
    // per split); the partials cost their write and read-back (at about 6 TB/s).  This
    // fills the GPU for skinny outputs (r x nrhs) and evens out the last wave of large ones.
    int nsm = 0;
    BEM_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const int T = mt * nt * nz;
    const int nch = (p.nkb + TC_CHUNK_KB - 1) / TC_CHUNK_KB;
    const double chunk_ms = (double)(Sg * (Sg + 1) / 2) * TC_CHUNK_KB * (TC_BK / 16) * 73.0 / 2.0e6 * BN / 128.0;
    // bytes per output per split written and read back: complex partials, or the real products
    const double part_ms_per_split = (double)p.Ml * p.ml * (zb ? 16.0 * nz : 32.0) / 6.0e9;
    int splits = 1;
    if (want_split >= 1) {
        // the stage's split count (at most one K' chunk per split, no empty splits)
        const int cps = (nch + std::min(want_split, nch) - 1) / std::min(want_split, nch);
        splits = (nch + cps - 1) / cps;
        if (splits > 1) p.kps = cps * TC_CHUNK_KB;
    } else {
        double best = (double)((T + nsm - 1) / nsm) * nch * chunk_ms;
        for (int s = 2; s <= 32 && s <= nch / 2; ++s) {
            const int cps = (nch + s - 1) / s;
            const int sr = (nch + cps - 1) / cps;
            if (sr != s) continue;
            const double cost = (double)(((int64_t)T * s + nsm - 1) / nsm) * cps * chunk_ms + s * part_ms_per_split;
            if (cost < 0.98 * best) { best = cost; splits = s; p.kps = cps * TC_CHUNK_KB; }
        }
    }
    if (zb) {
        const size_t need = (size_t)nz * splits * p.Ml * p.ml * sizeof(double);
        if (need > t->zbuf_cap) {
            if (t->zbuf) { cudaStreamSynchronize(h->stream); bem_dfree(h, t->zbuf); t->zbuf = nullptr; t->zbuf_cap = 0; }
            BEM_CUDA(h, bem_dmalloc(h, (void**)&t->zbuf, need));
            t->zbuf_cap = need;
        }
        p.outr = t->zbuf;
    } else if (splits > 1) {
        const size_t need = (size_t)splits * p.Ml * p.ml * sizeof(double2);
        if (need > t->part_cap) {
            if (t->part) { cudaStreamSynchronize(h->stream); bem_dfree(h, t->part); t->part = nullptr; t->part_cap = 0; }
            BEM_CUDA(h, bem_dmalloc(h, (void**)&t->part, need));
            t->part_cap = need;
        }
        p.part = t->part;
    }
    dim3 grid((unsigned)(mt * nt), (unsigned)splits, (unsigned)nz);
    BEM_TIMED(h, tag, (kern<<<grid, TC_THREADS, smem, h->stream>>>(A.map, mapB, p)));
    BEM_LAUNCH(h, "k_tc_gemm");
    if (zb) {
        if (transposed) {
            const dim3 cgrid((unsigned)((p.Ml + 31) / 32), (unsigned)((p.ml + 31) / 32));
            BEM_TIMED(h, "k_combine_blocks", (k_combine_blocks<<<cgrid, dim3(32, 8), 0, h->stream>>>(
                                                 p.outr, splits, zb->gauss, p.Ml, p.ml, out, ldo,
                                                 transposed, alpha, beta)));
        } else {
            const int64_t pairs = ((int64_t)p.Ml * p.ml + 1) / 2;
            BEM_TIMED(h, "k_combine_blocks", (k_combine_blocks_flat<<<(unsigned)((pairs + 255) / 256), 256, 0, h->stream>>>(
                                                 p.outr, splits, zb->gauss, p.Ml, p.ml, out, ldo, alpha, beta)));
        }
        BEM_LAUNCH(h, "k_combine_blocks");
        return BEM_OK;
    }
    if (splits > 1) {
        const int64_t n = (int64_t)p.Ml * p.ml;
        BEM_TIMED(h, "k_splitk_reduce", (k_splitk_reduce<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
                                            p.part, splits, p.Ml, p.ml, out, ldo, transposed, alpha, beta)));
        BEM_LAUNCH(h, "k_splitk_reduce");
    }
    return BEM_OK;
}

// ------------------------------------------------------------------------------ interface
// digit slices of the right-hand-side product (bem_options.rhs_slices; default one fewer
// than the operands hold)
static int rhs_slices(bem_ctx* h) {
    const int S = tcs(h)->S;
    const int Sr = h->opt.rhs_slices;
    return (Sr < 3 || Sr > S) ? std::max(3, S - 1) : Sr;
}

bem_status tc_prepare_operators(bem_ctx* h) {
    TcState* t = tcs(h);
    const int64_t N = h->N;
    bem_status st;
    // slices of X^T: row i of the A operand is column i of X (contiguous); row exponents
    // from the assembly when it gathered them.  S and N as row blocks [Re; Im; Re + Im]:
    // their products with complex factors (S Y with the right-hand sides, Y2 N in the
    // filter) then take Gauss's three real products instead of four, for one more block
    // written here (S's with the right-hand-side product's slices only); Q^T S takes S's
    // Re and Im blocks.  D keeps the part rows: it only meets the real Q^T.
    const int* fS = h->rexp_valid ? h->rexp : nullptr;
    const int* fW = h->rexp_valid ? h->rexp + N : nullptr;
    if ((st = slice_A(h, t->opS, h->S, N, N, N, 1, -1, 0, 0, fS, 3, rhs_slices(h))) != BEM_OK) return st;
    // N's near band (entries up to ~1e4 x its far field) is applied apart in double-float,
    // so the split only carries the far part with its own, much smaller row scale
    if ((st = slice_A(h, t->opW, h->W, N, N, N, 1, (int)std::min<int64_t>(TC_W_BAND, (N - 1) / 2), 0, 0, fW, 3,
                      t->S)) != BEM_OK)
        return st;
    if (h->D) {
        if ((st = slice_A(h, t->opD, h->D, N, N, N, 1)) != BEM_OK) return st;
    }
    return BEM_OK;
}

// out (nc x N, ld nc) += Y (nc x N, ld nc) * W_band, W_band = entries of W with cyclic
// |k - j| <= band; products and sums in double-float (about 48 bits) on the FP32 pipe.
// Tiled: a CTA owns 32 rows m and BAND_JB columns j; the Y rows it needs (k within the band
// of its columns) and the band of those W columns are converted to double-float once and
// staged in shared memory (Y as [k][m], so the 32 lanes read consecutive entries; W is
// read by all lanes of a warp at once).  Each thread accumulates BAND_JB/8 outputs.
#define BAND_JB 32
__global__ void __launch_bounds__(256, 1) k_band_left(const double2* __restrict__ Y, const double2* __restrict__ W,
                                                      int64_t N, int64_t nc, int band, double2* out) {
    extern __shared__ float4 bsm[];
    const int KT = BAND_JB + 2 * band;                 // k rows of the Y tile
    float4* Ys = bsm;                                   // [KT][32]
    float4* Ws = bsm + (size_t)KT * 32;                 // [BAND_JB][2 band + 1]
    const int64_t m0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * BAND_JB;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // cyclic indices wrapped by adding or subtracting N (one step when N exceeds the tile's
    // reach, a few for the smallest N); four iterations unrolled so their loads are in
    // flight together
#pragma unroll 4
    for (int idx = tid; idx < KT * 32; idx += 256) {
        const int kk = idx / 32, ml = idx % 32;
        int64_t k = j0 - band + kk;
        while (k < 0) k += N;
        while (k >= N) k -= N;
        const int64_t m = m0 + ml;
        double2 y = make_double2(0.0, 0.0);
        if (m < nc) y = Y[m + k * nc];
        Ys[idx] = cdfl_pack({dfl_from_bits(y.x), dfl_from_bits(y.y)});
    }
    const int BW = 2 * band + 1;
#pragma unroll 4
    for (int idx = tid; idx < BAND_JB * BW; idx += 256) {
        const int jl = idx / BW, t = idx % BW;
        const int64_t j = j0 + jl;
        double2 w = make_double2(0.0, 0.0);
        if (j < N) {
            int64_t k = j - band + t;
            while (k < 0) k += N;
            while (k >= N) k -= N;
            w = W[k + j * N];
        }
        Ws[idx] = cdfl_pack({dfl_from_bits(w.x), dfl_from_bits(w.y)});
    }
    __syncthreads();
    // each thread accumulates its BAND_JB / 8 outputs (columns jj = threadIdx.y + 8 i)
    // together, so their independent double-float chains hide each other's latency
    constexpr int NJ = BAND_JB / 8;
    const int ml = threadIdx.x;
    const int64_t m = m0 + ml;
    cdfl acc[NJ];
#pragma unroll
    for (int i = 0; i < NJ; ++i) acc[i] = cdfl_zero();
    for (int t = 0; t < BW; ++t) {
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            const int jj = threadIdx.y + 8 * i;
            const cdfl y = cdfl_unpack(Ys[(jj + t) * 32 + ml]);
            const cdfl w = cdfl_unpack(Ws[jj * BW + t]);
            acc[i].re = dfl_fma(y.re, w.re, dfl_fma(dfl_neg(y.im), w.im, acc[i].re));
            acc[i].im = dfl_fma(y.re, w.im, dfl_fma(y.im, w.re, acc[i].im));
        }
    }
#pragma unroll
    for (int i = 0; i < NJ; ++i) {
        const int64_t j = j0 + threadIdx.y + 8 * i;
        if (m < nc && j < N) {
            double2* o = out + m + j * nc;
            *o = cadd(*o, cdfl_to(acc[i]));
        }
    }
}

static const TcOperand* op_of(TcState* t, int op) {
    return op == TC_OP_S ? &t->opS : (op == TC_OP_W ? &t->opW : &t->opD);
}

bem_status tc_product_left(bem_ctx* h, int op, const double* Qreal, const cplx* Y, int64_t nc, cplx* out) {
    TcState* t = tcs(h);
    const int64_t N = h->N;
    const TcOperand* A = op_of(t, op);
    if (!A->slices) return bem_fail(h, BEM_E_INVALID, "tc_product_left: operator not sliced");
    bem_status st;
    // out^T = X^T L^T: B = Q (N x nc real) or Y^T (B[k, j] = Y[j + k nc]); a blocked A takes
    // two real products with the real Q (its Re and Im blocks), Gauss's three with Y^T
    if (Qreal) st = slice_B(h, t->bbuf, Qreal, 1, N, nc, 1, N);
    else st = slice_B(h, t->bbuf, Y, 0, N, nc, nc, 1, 0, A->blocks ? 3 : 0);
    if (st != BEM_OK) return st;
    const TcBlocks zr = {2, {0, 1, 0}, {0, 0, 0}, 0}, zg = {3, {0, 1, 2}, {0, 1, 2}, 1};
    st = tc_gemm(h, *A, t->bbuf, out, nc, 1, 1.0, 0.0,
                 op == TC_OP_S ? "tc_filter_QtS" : (op == TC_OP_W ? "tc_filter_YN" : "tc_filter_QtD"), 0,
                 A->blocks ? (Qreal ? &zr : &zg) : nullptr);
    if (st != BEM_OK || op != TC_OP_W) return st;
    if (!Y) return bem_fail(h, BEM_E_INVALID, "tc_product_left: N needs a complex left factor");
    const int band = (int)std::min<int64_t>(TC_W_BAND, (N - 1) / 2);
    dim3 grid((unsigned)((nc + 31) / 32), (unsigned)((N + BAND_JB - 1) / BAND_JB));
    const size_t bsmem = sizeof(float4) * ((size_t)(BAND_JB + 2 * band) * 32 + (size_t)BAND_JB * (2 * band + 1));
    BEM_CUDA(h, cudaFuncSetAttribute(k_band_left, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
    BEM_TIMED(h, "k_band_left", (k_band_left<<<grid, dim3(32, 8), bsmem, h->stream>>>(Y, h->W, N, nc, band, out)));
    BEM_LAUNCH(h, "k_band_left");
    return BEM_OK;
}

bem_status tc_product_right(bem_ctx* h, int op, const cplx* y, int64_t ldy, int64_t nrhs, cplx* out, int64_t ld) {
    TcState* t = tcs(h);
    const TcOperand* A = op_of(t, op);
    if (!A->slices) return bem_fail(h, BEM_E_INVALID, "tc_product_right: operator not sliced");
    // the right-hand sides take one digit slice fewer by default (see bem_options.rhs_slices);
    // a blocked A (S) takes Gauss's three real products
    const int Sr = rhs_slices(h);
    TcOperand& Bop = h->rhs_aux ? t->bbuf_rhs : t->bbuf;
    bem_status st = slice_B(h, Bop, y, 0, h->N, nrhs, 1, ldy, Sr, A->blocks ? 3 : 0);
    if (st != BEM_OK) return st;
    const TcBlocks zg = {3, {0, 1, 2}, {0, 1, 2}, 1};
    return tc_gemm(h, *A, Bop, out, ld, 0, 1.0, 0.0, "tc_rhs_SY", Sr, A->blocks ? &zg : nullptr);
}

bem_status tc_prepare_solve(bem_ctx* h) {
    TcState* t = tcs(h);
    const int64_t N = h->N, r = h->r;
    bem_status st;
    // V^H as A (r x N): A_op[i, k] = Vh[i + k r];  U as A (N x r): A_op[i, k] = U[i + k N]
    if ((st = slice_A(h, t->opVh, h->Vh, r, N, 1, r)) != BEM_OK) return st;
    return slice_A(h, t->opU, h->U, N, r, 1, N);
}

bem_status tc_compress_factors(bem_ctx* h, const double* Qs, cplx* U, cplx* Vh) {
    TcState* t = tcs(h);
    const int64_t N = h->N, nc = h->ncols, r = h->r;
    bem_status st;
    // U (N x r) = Qs (N x nc, real) E_r (nc x r)
    if ((st = slice_A(h, t->tmpA, Qs, N, nc, 1, N, -1, 1, 0)) != BEM_OK) return st;
    if ((st = slice_B(h, t->bbuf, h->E, 0, nc, r, 1, nc)) != BEM_OK) return st;
    if ((st = tc_gemm(h, t->tmpA, t->bbuf, U, N, 0, 1.0, 0.0, "tc_compress_U")) != BEM_OK) return st;
    // V^H (r x N) = E_r^H (r x nc) Bs (nc x N):  A_op[i, k] = conj(E[k + i nc])
    if ((st = slice_A(h, t->tmpA, h->E, r, nc, nc, 1, -1, 0, 1)) != BEM_OK) return st;
    if ((st = slice_B(h, t->bbuf, h->Bs, 0, nc, N, 1, nc)) != BEM_OK) return st;
    return tc_gemm(h, t->tmpA, t->bbuf, Vh, r, 0, 1.0, 0.0, "tc_compress_Vh");
}

bem_status tc_core_product(bem_ctx* h, cplx* Kt) {
    TcState* t = tcs(h);
    const int64_t N = h->N, r = h->r;
    if (!t->opVh.slices) return bem_fail(h, BEM_E_INVALID, "tc_core_product: call tc_prepare_solve first");
    // Kt = beta^-1 V^H U: A = V^H (sliced), B = U (N x r, column-major)
    bem_status st = slice_B(h, t->bbuf, h->U, 0, N, r, 1, N);
    if (st != BEM_OK) return st;
    return tc_gemm(h, t->opVh, t->bbuf, Kt, r, 0, 1.0 / h->beta, 0.0, "tc_factor_VhU");
}

// x = v/beta - beta^-2 U Kinv V^H v with tensor-core products (T, T2: r x nrhs scratch)
// Ss: digit slices of the two products (the leading Ss of U's and V^H's, v and T2 sliced
// with Ss), 0 = all of them
static bem_status woodbury_tc(bem_ctx* h, const cplx* v, int64_t ldv, cplx* x, int64_t ldx, int64_t nrhs, cplx* T,
                              cplx* T2, double xscale, double vscale, int Ss) {
    TcState* t = tcs(h);
    const int64_t N = h->N, r = h->r;
    bem_status st;
    if ((st = slice_B(h, t->bbuf, v, 0, N, nrhs, 1, ldv, Ss)) != BEM_OK) return st;
    if ((st = tc_gemm(h, t->opVh, t->bbuf, T, r, 0, 1.0, 0.0, "tc_solve_Vhv", Ss)) != BEM_OK) return st;
    h->tag = "gemm_solve_core";
    if ((st = zgemm_df(h, r, nrhs, r, h->K, r, T, r, T2, r)) != BEM_OK) return st;
    // x <- xscale x + vscale v / beta ; then x -= beta^-2 U T2
    if ((st = launch_axpby(h, x, ldx, v, ldv, cmk(vscale / h->beta, 0), cmk(xscale, 0), N, nrhs)) != BEM_OK) return st;
    if ((st = slice_B(h, t->bbuf, T2, 0, r, nrhs, 1, r, Ss)) != BEM_OK) return st;
    return tc_gemm(h, t->opU, t->bbuf, x, ldx, 0, -vscale / (h->beta * h->beta), 1.0, "tc_solve_UT", Ss);
}

bem_status tc_solve_refined(bem_ctx* h, const cplx* v, int64_t ldv, cplx* x, int64_t ldx, int64_t nrhs, int32_t* iters,
                            double* max_rel_resid) {
    TcState* t = tcs(h);
    const int64_t N = h->N, r = h->r;
    cplx *T = nullptr, *T2 = nullptr, *rho = nullptr;
    double* dres = nullptr;
    bem_status st;
    {
        void* base = nullptr;
        const size_t bT = ((sizeof(cplx) * r * nrhs + 255) / 256) * 256;
        const size_t bR = ((sizeof(cplx) * N * nrhs + 255) / 256) * 256;
        if ((st = bem_workspace(h, 2 * bT + bR + 256, &base)) != BEM_OK) return st;
        T = (cplx*)base;
        T2 = (cplx*)((char*)base + bT);
        rho = (cplx*)((char*)base + 2 * bT);
        dres = (double*)((char*)base + 2 * bT + bR);
    }
    // the Woodbury solves (initial and corrections) may use fewer digit slices than the
    // residual products (bem_options.solve_slices); the refinement then recovers the digits
    int Ss = h->opt.solve_slices;
    if (Ss < 3 || Ss > t->S) Ss = 0;
    // initial solve
    if ((st = woodbury_tc(h, v, ldv, x, ldx, nrhs, T, T2, 0.0, 1.0, Ss)) != BEM_OK) return st;
    int it = 0;
    double res = 0.0;
    for (;;) {
        // rho = v - (beta x + U V^H x)
        if ((st = slice_B(h, t->bbuf, x, 0, N, nrhs, 1, ldx)) != BEM_OK) return st;
        if ((st = tc_gemm(h, t->opVh, t->bbuf, T, r, 0, 1.0, 0.0, "tc_resid_Vhx")) != BEM_OK) return st;
        if ((st = launch_copy2d(h, rho, N, v, ldv, N, nrhs, sizeof(cplx))) != BEM_OK) return st;
        if ((st = launch_axpby(h, rho, N, x, ldx, cmk(-h->beta, 0), cmk(1, 0), N, nrhs)) != BEM_OK) return st;
        if ((st = slice_B(h, t->bbuf, T, 0, r, nrhs, 1, r)) != BEM_OK) return st;
        if ((st = tc_gemm(h, t->opU, t->bbuf, rho, N, 0, -1.0, 1.0, "tc_resid_UT")) != BEM_OK) return st;
        if ((st = launch_col_norm_ratio(h, rho, N, v, ldv, N, nrhs, dres)) != BEM_OK) return st;
        int e = 0;
        BEM_CUDA(h, cudaMemcpyAsync(&res, dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        BEM_CUDA(h, cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        BEM_CUDA(h, cudaStreamSynchronize(h->stream));   // this stream only (not the whole device)
        if (e) {
            cudaMemset(h->dev_err, 0, sizeof(int));
            return bem_fail(h, (e & DEVERR_TIMEOUT) ? BEM_E_TIMEOUT : BEM_E_CUDA, "tensor-core solve: device error");
        }
        if (!(res > h->opt.refine_rtol) || it >= h->opt.max_refine) break;
        // x += Woodbury(rho)
        if ((st = woodbury_tc(h, rho, N, x, ldx, nrhs, T, T2, 1.0, 1.0, Ss)) != BEM_OK) return st;
        ++it;
    }
    if (iters) *iters = it;
    if (max_rel_resid) *max_rel_resid = res;
    if (res > h->opt.refine_rtol || res != res)
        return bem_fail(h, BEM_E_NOT_CONVERGED, "mixed solve: residual " + std::to_string(res) + " above refine_rtol");
    return BEM_OK;
}

static void free_op(bem_ctx* h, TcOperand& op) {
    bem_dfree(h, op.slices);
    bem_dfree(h, op.exps);
    op = TcOperand();
}

void tc_release_operands(bem_ctx* h) {
    if (!h->tc) return;
    TcState* t = (TcState*)h->tc;
    free_op(h, t->opS); free_op(h, t->opW); free_op(h, t->opD);
}
void tc_release_solve(bem_ctx* h) {
    if (!h->tc) return;
    TcState* t = (TcState*)h->tc;
    free_op(h, t->opVh); free_op(h, t->opU);
}
void tc_destroy(bem_ctx* h) {
    if (!h->tc) return;
    TcState* t = (TcState*)h->tc;
    free_op(h, t->opS); free_op(h, t->opW); free_op(h, t->opD); free_op(h, t->opVh); free_op(h, t->opU);
    free_op(h, t->bbuf);
    free_op(h, t->bbuf_rhs);
    free_op(h, t->tmpA);
    bem_dfree(h, t->part);
    bem_dfree(h, t->zbuf);
    delete t;
    h->tc = nullptr;
}
