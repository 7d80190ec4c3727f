// Double-float arithmetic: unevaluated sums hi + lo of two floats (about 48 significant
// bits).  GB300 issues FP32 at 64x its FP64 rate, so FP64-accurate work that is bound by
// arithmetic (the far-field assembly, the mixed path's QR) runs in this form on the FP32
// pipe.  Dekker's product via fmaf and Knuth's two-sum; the _rn intrinsics keep the
// compiler from contracting or reassociating the error terms.  Accuracy is relative to the
// operands' magnitudes.
#pragma once

#include "common.cuh"

struct dfl { float hi, lo; };
struct cdfl { dfl re, im; };

__device__ __forceinline__ dfl dfl_mk(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ dfl dfl_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
// exact float -> double by moving the bit fields (the FP64 pipe's conversion is as slow as
// its arithmetic); subnormal floats become zero
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 255u;
    if (e == 0u) return 0.0;
    const unsigned hiw = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hiw, (int)(u << 29));
}
__device__ __forceinline__ double dfl_to(dfl a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }
// double -> double-float from the bit fields (integer operations and one int-to-float
// conversion): hi = the significand rounded to 24 bits, lo = the remainder (<= 29 bits,
// rounded to 24).  |x| must lie in the float normal range or be below 2^-74 (-> 0).
__device__ __forceinline__ dfl dfl_from_bits(double x) {
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E < 949 || E > 1149) return {0.f, 0.f};
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    long long m24 = (m + (1LL << 28)) >> 29;              // 24-bit significand, rounded
    const int rem = (int)(m - (m24 << 29));                // |rem| <= 2^28
    int eh = E;
    if (m24 == (1LL << 24)) { m24 >>= 1; ++eh; }
    const unsigned sgn = (unsigned)((unsigned long long)b >> 63) << 31;
    const float hi = __uint_as_float(sgn | ((unsigned)(eh - 896) << 23) | ((unsigned)m24 & 0x7FFFFFu));
    float lo = __int2float_rn(rem) * __uint_as_float((unsigned)(E - 1075 + 127) << 23);
    if (sgn) lo = -lo;
    return {hi, lo};
}
__device__ __forceinline__ dfl dfl_qts(float s, float e) {    // |s| >= |e|
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return dfl_qts(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl dfl_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl dfl_sub(dfl a, dfl b) { return dfl_add(a, dfl_neg(b)); }
__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dfl_qts(p, e);
}
// a * b + c
__device__ __forceinline__ dfl dfl_fma(dfl a, dfl b, dfl c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    const float s = __fadd_rn(p, c.hi);
    const float bb = __fsub_rn(s, p);
    const float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
    return dfl_qts(s, __fadd_rn(e, __fadd_rn(pe, c.lo)));
}
__device__ __forceinline__ dfl dfl_scale(dfl a, float p2) { return {a.hi * p2, a.lo * p2}; }   // p2 a power of 2
__device__ __forceinline__ cdfl cdfl_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cdfl cdfl_add(cdfl a, cdfl b) { return {dfl_add(a.re, b.re), dfl_add(a.im, b.im)}; }
__device__ __forceinline__ cdfl cdfl_sub(cdfl a, cdfl b) { return {dfl_sub(a.re, b.re), dfl_sub(a.im, b.im)}; }
__device__ __forceinline__ cdfl cdfl_scale(dfl w, cdfl g) { return {dfl_mul(w, g.re), dfl_mul(w, g.im)}; }   // w g
__device__ __forceinline__ cdfl cdfl_fma_real(dfl w, cdfl g, cdfl acc) {   // w g + acc
    return {dfl_fma(w, g.re, acc.re), dfl_fma(w, g.im, acc.im)};
}
__device__ __forceinline__ cdfl cdfl_from(cplx z) { return {dfl_from(z.x), dfl_from(z.y)}; }
__device__ __forceinline__ cplx cdfl_to(cdfl z) { return cmk(dfl_to(z.re), dfl_to(z.im)); }
__device__ __forceinline__ float4 cdfl_pack(cdfl z) { return make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo); }
__device__ __forceinline__ cdfl cdfl_unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }


// Fixed point: exact sums and differences of double-floats of one scale.
// round(v 2^sh) of a float as a 64-bit integer, from its bit fields (the caller keeps
// |v| 2^sh below 2^62; bits below 2^-sh are rounded off)
__device__ __forceinline__ long long f32_to_fixed(float v, int sh) {
    const int b = __float_as_int(v);
    const int ex = (b >> 23) & 255;
    if (ex == 0) return 0;
    const long long m = (long long)((b & 0x7FFFFF) | 0x800000);
    const int s = ex - 150 + sh;                            // v = m 2^(ex - 150)
    long long r;
    if (s >= 0) r = m << s;
    else if (s >= -25) r = (m + (1LL << (-s - 1))) >> (-s);
    else r = 0;
    return b < 0 ? -r : r;
}
__device__ __forceinline__ long long dfl_to_fixed(dfl a, int sh) { return f32_to_fixed(a.hi, sh) + f32_to_fixed(a.lo, sh); }
// v 2^-sh as a double, rounded to nearest (ties to even), from the bit fields (integer
// operations only); results below the double normal range become 0
__device__ __forceinline__ double fixed_to_double(long long v, int sh) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = v < 0 ? (1ULL << 63) : 0ULL;
    unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll((long long)u);
    u <<= lz;                                               // bit 63 set: value u 2^(-lz - sh)
    unsigned long long m = u >> 11;                         // 53 bits, bit 52 set
    const unsigned long long rest = u & 0x7FFULL;
    int E = 63 - lz - sh;
    if (rest > 0x400ULL || (rest == 0x400ULL && (m & 1ULL))) {
        ++m;
        if (m == (1ULL << 53)) { m >>= 1; ++E; }
    }
    if (E + 1023 < 1) return 0.0;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(E + 1023) << 52) | (m & ((1ULL << 52) - 1))));
}

// sqrt, 1/sqrt and division with one Newton correction of the float estimate (about 47
// bits); arguments in the float normal range, x > 0 for the roots
__device__ __forceinline__ dfl dfl_sqrt(dfl x) {
    const float y = sqrtf(x.hi);
    const dfl y2 = dfl_mul(dfl{y, 0.f}, dfl{y, 0.f});
    const dfl r = dfl_sub(x, y2);
    return dfl_qts(y, r.hi * (0.5f / y));
}
__device__ __forceinline__ dfl dfl_rsqrt(dfl x) {
    const float y = rsqrtf(x.hi);
    // y' = y + y (1 - x y^2) / 2
    const dfl xy = dfl_mul(x, dfl{y, 0.f});
    const dfl r = dfl_sub(dfl{1.f, 0.f}, dfl_mul(xy, dfl{y, 0.f}));
    return dfl_qts(y, y * 0.5f * r.hi);
}
__device__ __forceinline__ dfl dfl_div(dfl a, dfl b) {
    const float q = a.hi / b.hi;
    const dfl r = dfl_sub(a, dfl_mul(dfl{q, 0.f}, b));
    return dfl_qts(q, r.hi / b.hi);
}
