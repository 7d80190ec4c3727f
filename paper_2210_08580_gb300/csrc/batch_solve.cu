// Grouped FP64 Woodbury solve of many factored problems in ONE persistent launch: the solve
// stage of the batching layer (the paper solves one geometry at a time; the solve itself is
// the Woodbury form of the compressed operator, Sec. IV-C):
//     x_p = v_p / beta_p - beta_p^-2 U_p Kinv_p (V_p^H v_p)      for every problem p.
// Three stages of 64 x 64 complex tiles (column-major, FP64 FMAs) taken from one global
// queue by persistent CTAs:
//     A  partial products V^H v over 256-long slices of N (split K: every SM gets work even
//        when each problem has a handful of right-hand-side blocks, and a problem's chain of
//        stages stays short: 16 K steps per slice instead of N/16); above N = 16384 the
//        slices lengthen to ceil(N / 64), rounded up to 16, so that no problem keeps more
//        than 64 partial products (the slicing depends on the problem's own N only),
//     B  T2 = Kinv T, with T summed from the slices in slice order (a fixed order: the
//        result does not depend on which CTA ran what),
//     C  x = v / beta - beta^-2 U T2.
// The queue hands out every A tile before any B tile and every B tile before any C tile, so
// a tile only ever waits for tiles that running CTAs have already taken: no deadlock,
// whatever the residency.  Per problem and column block a counter records the finished A
// tiles (B waits on it) and the finished B tiles (C waits on it); the waits are bounded in
// wall time (10 s, against about 1 ms in a normal run) and set DEVERR_TIMEOUT when they give
// up, after which every CTA stops taking tiles and the call returns BEM_E_TIMEOUT.
#include <algorithm>
#include <numeric>
#include <vector>

#include "kernels.h"

#define WB_T 64      // tile edge (rows and right-hand sides)
#define WB_BK 16     // K step staged in shared memory
#define WB_KC 256    // slice of N per stage-A tile (at least)
#define WB_NCH 64    // most slices per problem

struct WbProb {
    const cplx* U;       // N x r, ld N
    const cplx* Vh;      // r x N, ld r
    const cplx* K;       // r x r, ld r (the inverted Woodbury core)
    const cplx* v;       // N x nrhs, ld ldv
    cplx* x;             // N x nrhs, ld ldx
    cplx* part;          // nch slices of r x nrhs (ld r)
    cplx* T2;            // r x nrhs (ld r)
    int* cnt;            // [0, ncb): A tiles done per column block; [ncb, 2 ncb): B tiles done
    long long ldv, ldx;
    long long first[3];  // first tile of this problem in each stage's range
    int N, r, nrhs, mr, ncb, nch, mN, kc;
    double ib, c2;       // 1 / beta and -1 / beta^2
};

__device__ __forceinline__ int wb_ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// acc (4 x 4 complex per thread: rows tx + 16 i, columns ty + 16 j of the tile) +=
// A[m0.., kbeg..kend) * B[kbeg..kend), n0..), A column-major (lda, M rows), B through loadB.
template <class LoadB>
__device__ __forceinline__ void wb_tile(cplx (&acc)[4][4], const cplx* __restrict__ A, long long lda, int M,
                                        int m0, int kbeg, int kend, LoadB loadB, cplx (*As)[WB_T],
                                        cplx (*Bs)[WB_T]) {
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    for (int k0 = kbeg; k0 < kend; k0 += WB_BK) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int mm = t % 64, kk = t / 64 + 4 * s;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < kend) ? A[gm + (long long)gk * lda] : cmk(0, 0);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int kk = t % 16, nn = t / 16 + 16 * s;
            const int gk = k0 + kk;
            Bs[kk][nn] = (gk < kend) ? loadB(gk, nn) : cmk(0, 0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < WB_BK; ++kk) {
            cplx a[4], b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned long long wb_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 waits until *c >= target, for at most limit_ns of wall time (the global timer;
// a spin count caps it as well); false when the wait gave up (DEVERR_TIMEOUT) or another
// CTA reported an error.  Every thread returns the same value.
__device__ __forceinline__ bool wb_wait(const int* c, int target, int* err, int* s_ok,
                                        unsigned long long limit_ns) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = wb_globaltimer();
        for (long long spins = 0; wb_ld_acquire(c) < target; ++spins) {
            if ((spins & 63) == 63) {
                if (*(volatile int*)err) { ok = 0; break; }
                if (wb_globaltimer() - t0 > limit_ns || spins > (1ll << 26)) {
                    atomicOr(err, DEVERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
            if (spins > 32) __nanosleep(128);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// This CTA's writes of the tile, then one arrival on *c.
__device__ __forceinline__ void wb_signal(int* c) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(c, 1);
    }
}

__global__ void __launch_bounds__(256) k_woodbury_batch(const WbProb* __restrict__ ps, int nprob,
                                                        long long nA, long long nB, long long nC,
                                                        unsigned long long* queue, int* err,
                                                        unsigned long long limit_ns) {
    __shared__ cplx As[WB_BK][WB_T];
    __shared__ cplx Bs[WB_BK][WB_T];
    __shared__ long long s_t;
    __shared__ int s_p, s_ok;
    const long long total = nA + nB + nC;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    for (;;) {
        __syncthreads();
        if (t == 0) {
            long long q = (long long)atomicAdd(queue, 1ull);
            if (*(volatile int*)err) q = total;
            s_t = q;
            if (q < total) {
                const int stage = q < nA ? 0 : (q < nA + nB ? 1 : 2);
                const long long loc = q - (stage == 0 ? 0 : (stage == 1 ? nA : nA + nB));
                int lo = 0, hi = nprob - 1;          // last problem whose first tile <= loc
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (ps[mid].first[stage] <= loc) lo = mid; else hi = mid - 1;
                }
                s_p = lo;
            }
        }
        __syncthreads();
        const long long q = s_t;
        if (q >= total) break;
        const WbProb& P = ps[s_p];
        cplx acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = cmk(0, 0);
        if (q < nA) {
            // A: tile (rb, cb) of slice c of V^H v
            long long l = q - P.first[0];
            const int rb = (int)(l % P.mr);
            l /= P.mr;
            const int c = (int)(l % P.nch);
            const int cb = (int)(l / P.nch);
            const int m0 = rb * WB_T, n0 = cb * WB_T;
            const int kbeg = c * P.kc, kend = min(P.N, kbeg + P.kc);
            const cplx* v = P.v;
            const long long ldv = P.ldv;
            const int nrhs = P.nrhs;
            wb_tile(acc, P.Vh, P.r, P.r, m0, kbeg, kend,
                    [=](int gk, int nn) { const int gn = n0 + nn;
                                          return gn < nrhs ? v[gk + (long long)gn * ldv] : cmk(0, 0); },
                    As, Bs);
            cplx* out = P.part + (long long)c * P.r * P.nrhs;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gm = m0 + tx + 16 * i;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gn = n0 + ty + 16 * j;
                    if (gm < P.r && gn < P.nrhs) out[gm + (long long)gn * P.r] = acc[i][j];
                }
            }
            wb_signal(P.cnt + cb);
        } else if (q < nA + nB) {
            // B: tile (rb, cb) of T2 = Kinv T, T = sum of the slices in slice order
            const long long l = q - nA - P.first[1];
            const int rb = (int)(l % P.mr), cb = (int)(l / P.mr);
            if (!wb_wait(P.cnt + cb, P.mr * P.nch, err, &s_ok, limit_ns)) continue;
            const int m0 = rb * WB_T, n0 = cb * WB_T;
            const cplx* part = P.part;
            const long long slice = (long long)P.r * P.nrhs;
            const int nch = P.nch, r = P.r, nrhs = P.nrhs;
            wb_tile(acc, P.K, P.r, P.r, m0, 0, P.r,
                    [=](int gk, int nn) {
                        const int gn = n0 + nn;
                        cplx s = cmk(0, 0);
                        if (gn < nrhs) {
                            const cplx* p = part + gk + (long long)gn * r;
                            for (int c = 0; c < nch; ++c) {
                                const cplx w = __ldcg(p + c * slice);
                                s.x += w.x;
                                s.y += w.y;
                            }
                        }
                        return s;
                    },
                    As, Bs);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gm = m0 + tx + 16 * i;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gn = n0 + ty + 16 * j;
                    if (gm < P.r && gn < P.nrhs) P.T2[gm + (long long)gn * P.r] = acc[i][j];
                }
            }
            wb_signal(P.cnt + P.ncb + cb);
        } else {
            // C: tile (rb, cb) of x = v / beta - beta^-2 U T2
            const long long l = q - nA - nB - P.first[2];
            const int rb = (int)(l % P.mN), cb = (int)(l / P.mN);
            if (!wb_wait(P.cnt + P.ncb + cb, P.mr, err, &s_ok, limit_ns)) continue;
            const int m0 = rb * WB_T, n0 = cb * WB_T;
            const cplx* T2 = P.T2;
            const int r = P.r, nrhs = P.nrhs;
            wb_tile(acc, P.U, P.N, P.N, m0, 0, P.r,
                    [=](int gk, int nn) { const int gn = n0 + nn;
                                          return gn < nrhs ? __ldcg(T2 + gk + (long long)gn * r) : cmk(0, 0); },
                    As, Bs);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gm = m0 + tx + 16 * i;
                if (gm >= P.N) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gn = n0 + ty + 16 * j;
                    if (gn >= P.nrhs) continue;
                    const cplx vv = P.v[gm + (long long)gn * P.ldv];
                    P.x[gm + (long long)gn * P.ldx] =
                        cmk(fma(P.c2, acc[i][j].x, vv.x * P.ib), fma(P.c2, acc[i][j].y, vv.y * P.ib));
                }
            }
        }
    }
}

static size_t wb_align(size_t b) { return (b + 255) & ~(size_t)255; }

// stall_ms > 0: the failure-detection check (bem_solve_batch_stall_check): the first stage-A
// counter of the first problem in the queue starts far below its target, so the waits of that
// block's stage-B tiles give up after stall_ms (every wait then runs with that limit).
static bem_status solve_batch_impl(bem_handle* hs, int64_t nprob, const void* const* v_dev, const int64_t* ldv,
                                   void* const* x_dev, const int64_t* ldx, const int64_t* nrhs, int stall_ms) {
    if (!hs || !v_dev || !ldv || !x_dev || !ldx || !nrhs || nprob < 1 || nprob > 65536) return BEM_E_INVALID;
    for (int64_t q = 0; q < nprob; ++q)
        if (!hs[q]) return BEM_E_INVALID;
    bem_ctx* h0 = hs[0];
    for (int64_t q = 0; q < nprob; ++q) hs[q]->err.clear();
    auto fail = [&](int64_t q, bem_status st, const std::string& msg) {
        const std::string m = "bem_solve_batch: problem " + std::to_string(q) + ": " + msg;
        if (q > 0) bem_fail(hs[q], st, m);
        return bem_fail(h0, st, m);
    };
    for (int64_t q = 0; q < nprob; ++q) {
        const bem_ctx* h = hs[q];
        if (h->device != h0->device) return fail(q, BEM_E_INVALID, "every handle must be on the same device");
        if (h->stage < 4) return fail(q, BEM_E_INVALID, "call factor first");
        if (!v_dev[q] || !x_dev[q] || v_dev[q] == x_dev[q] || nrhs[q] < 1 || nrhs[q] > (1 << 24) ||
            ldv[q] < h->N || ldx[q] < h->N)
            return fail(q, BEM_E_INVALID, "need v, x (not aliased), 1 <= nrhs <= 2^24, ld >= N");
        if (h->N >= (int64_t)1 << 30) return fail(q, BEM_E_UNSUPPORTED, "N too large");
    }
    // problems with the most stage-A work first
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    auto work = [&](int q) { return (double)hs[q]->N * (double)hs[q]->r * (double)nrhs[q]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<WbProb> ps(nprob);
    long long tot[3] = {0, 0, 0};
    size_t cnt_ints = 0, scratch = 0;
    for (int64_t i = 0; i < nprob; ++i) {
        const int q = order[i];
        const bem_ctx* h = hs[q];
        WbProb& P = ps[i];
        P.U = h->U; P.Vh = h->Vh; P.K = h->K;
        P.v = (const cplx*)v_dev[q]; P.x = (cplx*)x_dev[q];
        P.ldv = ldv[q]; P.ldx = ldx[q];
        P.N = (int)h->N; P.r = (int)h->r; P.nrhs = (int)nrhs[q];
        P.mr = (P.r + WB_T - 1) / WB_T;
        P.ncb = (P.nrhs + WB_T - 1) / WB_T;
        P.kc = std::max(WB_KC, ((P.N + WB_NCH - 1) / WB_NCH + 15) / 16 * 16);
        P.nch = (P.N + P.kc - 1) / P.kc;
        P.mN = (P.N + WB_T - 1) / WB_T;
        P.ib = 1.0 / h->beta;
        P.c2 = -1.0 / (h->beta * h->beta);
        P.first[0] = tot[0]; tot[0] += (long long)P.mr * P.ncb * P.nch;
        P.first[1] = tot[1]; tot[1] += (long long)P.mr * P.ncb;
        P.first[2] = tot[2]; tot[2] += (long long)P.mN * P.ncb;
        cnt_ints += 2 * (size_t)P.ncb;
        scratch += wb_align(sizeof(cplx) * (size_t)P.r * P.nrhs * (P.nch + 1));
    }
    // one block: queue and counters (zeroed), then the problem table, then the scratch
    const size_t head = wb_align(sizeof(unsigned long long) + sizeof(int) * cnt_ints);
    const size_t table = wb_align(sizeof(WbProb) * nprob);
    void* buf = nullptr;
    cudaError_t e = cudaSetDevice(h0->device);
    if (e != cudaSuccess) return bem_cuda_check(h0, e, "bem_solve_batch: cudaSetDevice");
    if ((e = bem_dmalloc_async(h0, &buf, head + table + scratch)) != cudaSuccess)
        return bem_cuda_check(h0, e, "bem_solve_batch: scratch");
    unsigned long long* queue = (unsigned long long*)buf;
    int* cnt = (int*)((char*)buf + sizeof(unsigned long long));
    WbProb* dps = (WbProb*)((char*)buf + head);
    char* sp = (char*)buf + head + table;
    for (int64_t i = 0; i < nprob; ++i) {
        WbProb& P = ps[i];
        P.cnt = cnt;
        cnt += 2 * P.ncb;
        P.T2 = (cplx*)sp;
        P.part = P.T2 + (size_t)P.r * P.nrhs;
        sp += wb_align(sizeof(cplx) * (size_t)P.r * P.nrhs * (P.nch + 1));
    }
    // every handle's earlier work (its factors, its right-hand sides) before the launch
    std::vector<cudaEvent_t> evs;
    for (int64_t q = 1; q < nprob; ++q) {
        if (hs[q]->stream == h0->stream) continue;
        cudaEvent_t ev = bem_event_get(hs[q]);
        cudaEventRecord(ev, hs[q]->stream);
        cudaStreamWaitEvent(h0->stream, ev, 0);
        hs[q]->evpool.push_back(ev);
    }
    bem_status st = BEM_OK;
    e = cudaMemsetAsync(buf, 0, head, h0->stream);
    static const int k_stalled = -(1 << 30);
    if (e == cudaSuccess && stall_ms > 0)
        e = cudaMemcpyAsync(ps[0].cnt, &k_stalled, sizeof(int), cudaMemcpyHostToDevice, h0->stream);
    // a wait lasts about one stage-A tile (about 1 ms of one SM's FP64 pipe) in a normal run
    const unsigned long long limit_ns = stall_ms > 0 ? 1000000ull * (unsigned long long)stall_ms : 10000000000ull;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dps, ps.data(), sizeof(WbProb) * nprob, cudaMemcpyHostToDevice, h0->stream);
    int per = 0, nsm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_woodbury_batch, 256, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h0->device);
    if (e != cudaSuccess) st = bem_cuda_check(h0, e, "bem_solve_batch: launch setup");
    if (st == BEM_OK) {
        const long long all = tot[0] + tot[1] + tot[2];
        const long long ctas = std::min<long long>(all, (long long)std::max(per, 1) * nsm);
        BEM_TIMED(h0, "k_woodbury_batch", (k_woodbury_batch<<<(unsigned)ctas, 256, 0, h0->stream>>>(
                                              dps, (int)nprob, tot[0], tot[1], tot[2], queue, h0->dev_err,
                                              limit_ns)));
        e = cudaGetLastError();
        if (e != cudaSuccess) st = bem_cuda_check(h0, e, "k_woodbury_batch");
    }
    bem_dfree_async(h0, buf);
    // every handle's later work after it
    for (int64_t q = 1; q < nprob; ++q) {
        if (hs[q]->stream == h0->stream) continue;
        cudaEvent_t ev = bem_event_get(h0);
        cudaEventRecord(ev, h0->stream);
        cudaStreamWaitEvent(hs[q]->stream, ev, 0);
        h0->evpool.push_back(ev);
    }
    if (st != BEM_OK) return st;
    int flag = 0;
    e = cudaMemcpyAsync(&flag, h0->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h0->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h0->stream);
    if (e != cudaSuccess) return bem_cuda_check(h0, e, "bem_solve_batch: status");
    if (flag) {
        cudaMemsetAsync(h0->dev_err, 0, sizeof(int), h0->stream);
        if (flag & DEVERR_TIMEOUT) return bem_fail(h0, BEM_E_TIMEOUT, "bem_solve_batch: a device-side wait timed out");
        return bem_fail(h0, BEM_E_CUDA, "bem_solve_batch: device error flag set");
    }
    return BEM_OK;
}

extern "C" bem_status bem_solve_batch(bem_handle* hs, int64_t nprob, const void* const* v_dev, const int64_t* ldv,
                                      void* const* x_dev, const int64_t* ldx, const int64_t* nrhs) {
    return solve_batch_impl(hs, nprob, v_dev, ldv, x_dev, ldx, nrhs, 0);
}

extern "C" bem_status bem_solve_batch_stall_check(bem_handle* hs, int64_t nprob, const void* const* v_dev,
                                                  const int64_t* ldv, void* const* x_dev, const int64_t* ldx,
                                                  const int64_t* nrhs, int stall_ms) {
    if (stall_ms < 1 || stall_ms > 10000) return BEM_E_INVALID;
    return solve_batch_impl(hs, nprob, v_dev, ldv, x_dev, ldx, nrhs, stall_ms);
}
