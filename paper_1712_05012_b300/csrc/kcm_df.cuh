// Double-float arithmetic for the mixed-precision kinematics and torque kernels.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant
// bits. On B300 a float instruction retires 32 lanes per cycle per SM sub-partition while an FP64
// warp instruction takes about 84 cycles, so the ~10-20 float instructions of a double-float
// operation cost a fraction of one FP64 instruction, and their dependent latency (4 cycles each) is
// far below FP64's (~70). The error-free transforms are the classical ones (Knuth's two-sum, the
// fused-multiply-add two-product, Dekker's fast two-sum); every step uses an explicitly rounded
// intrinsic so that the compiler cannot contract or reorder it.
//
// The same kernels are compiled for double (FP64 mode) through the overloads at the end: for double
// the operations are the plain ones, in the order the FP64 kernels always used.
#pragma once

#include <cuda_runtime.h>

namespace kcm {
namespace dev {

struct df {
    float hi, lo;
};
static_assert(sizeof(df) == sizeof(double), "a double-float fills the slot of a double");

__device__ __forceinline__ df df_from(float x) { return {x, 0.0f}; }

// nearest double-float to a double (two FP64 conversions and one FP64 subtraction)
__device__ __forceinline__ df df_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(__dsub_rn(x, (double)h))};
}
__device__ __forceinline__ double to_double(df a) { return __dadd_rn((double)a.hi, (double)a.lo); }

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return {s, e};
}
// s + e = a + b exactly, for |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }
__device__ __forceinline__ df mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a * b + c
__device__ __forceinline__ df fma(df a, df b, df c) { return add(mul(a, b), c); }
// exact scaling by a power of two
__device__ __forceinline__ df ldexp2(df a, float p2) { return {__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }

// Exact double-float of an int64 x with |x| < 2^48 (larger values are rounded to about 2^-24
// relative): x = h 2^24 + l with h = x >> 24 (arithmetic) and 0 <= l < 2^24, both exact in float.
__device__ __forceinline__ df df_from_i64(long long x) {
    const float h = (float)(int)(x >> 24);
    const float l = (float)(int)(x & 0xFFFFFFLL);
    return two_sum(__fmul_rn(h, 16777216.0f), l);
}

// Order-preserving 64-bit key of a normalized double-float (hi = the float nearest to hi + lo, which the
// operations above keep): the order of the keys is the order of the values, and the key decodes to the
// same pair, so minima and maxima of exact double-float values need no FP64 arithmetic.
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k); }
__device__ __forceinline__ unsigned long long dfkey(df v) { return ((unsigned long long)fkey(v.hi) << 32) | fkey(v.lo); }
__device__ __forceinline__ df dfkey_inv(unsigned long long k) { return {fkey_inv((unsigned)(k >> 32)), fkey_inv((unsigned)k)}; }

__device__ __forceinline__ df shfl(df a, int src) {
    return {__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
}
__device__ __forceinline__ df shfl_up(df a, int off) {
    return {__shfl_up_sync(0xffffffffu, a.hi, off), __shfl_up_sync(0xffffffffu, a.lo, off)};
}
__device__ __forceinline__ df shfl_down(df a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.hi, off), __shfl_down_sync(0xffffffffu, a.lo, off)};
}

// sin and cos of a double angle as double-floats. Range reduction in FP64 by Cody and Waite's
// method: k = nearest integer to th * 2/pi, r = th - k (P1 + P2 + P3) with pi/2 split into a 33-bit,
// a second 33-bit and a remainder double, so k P1 and k P2 are exact for |k| < 2^20. Then the Taylor
// series of sin and cos in x = r^2 (|r| <= pi/4; the first omitted terms are below 5e-17), evaluated
// by Horner's rule in double-float, and the quadrant k mod 4.
struct df_sc {
    df s, c;
};
__device__ __forceinline__ df_sc df_sincos_v(double th) {
    // 1/n! as float pairs (hi + lo within 2e-16 relative of the exact rational)
    constexpr float kInvFact[18][2] = {
        {1.0f, 0.0f}, {1.0f, 0.0f}, {0x1p-1f, 0.0f},
        {0x1.555556p-3f, -0x1.555556p-28f}, {0x1.555556p-5f, -0x1.555556p-30f},
        {0x1.111112p-7f, -0x1.dddddep-32f}, {0x1.6c16c2p-10f, -0x1.27d27ep-35f},
        {0x1.a01a02p-13f, -0x1.7f97fap-39f}, {0x1.a01a02p-16f, -0x1.7f97fap-42f},
        {0x1.71de3ap-19f, 0x1.55b1ccp-45f}, {0x1.27e4fcp-22f, -0x1.10ec14p-47f},
        {0x1.ae6456p-26f, 0x1.fd5138p-52f}, {0x1.1eed8ep-29f, 0x1.ff1b12p-54f},
        {0x1.612462p-33f, -0x1.8af25ep-58f}, {0x1.93974ap-37f, 0x1.180f94p-62f},
        {0x1.ae7f3ep-41f, 0x1.ccee08p-67f}, {0x1.ae7f3ep-45f, 0x1.ccee08p-71f},
        {0x1.952c78p-49f, -0x1.f9ea56p-74f}};
    const double k = rint(th * 0x1.45f306dc9c883p-1);
    double r = ::fma(-k, 0x1.921fb544p+0, th);
    r = ::fma(-k, 0x1.0b4611a6p-34, r);
    r = ::fma(-k, 0x1.3198a2e037073p-69, r);
    const df rr = df_from(r);
    const df x = mul(rr, rr);
    // sin r = r (1 - x/3! + x^2/5! - ... - x^7/15!)
    df ps = {kInvFact[15][0], kInvFact[15][1]};
    ps = neg(ps);
#pragma unroll
    for (int n = 13; n >= 3; n -= 2) {
        const float sg = ((n - 1) / 2) % 2 ? -1.0f : 1.0f;
        ps = fma(ps, x, df{sg * kInvFact[n][0], sg * kInvFact[n][1]});
    }
    ps = fma(ps, x, df{1.0f, 0.0f});
    const df sr = mul(ps, rr);
    // cos r = 1 - x/2! + x^2/4! - ... + x^8/16!
    df pc = {kInvFact[16][0], kInvFact[16][1]};
#pragma unroll
    for (int n = 14; n >= 2; n -= 2) {
        const float sg = (n / 2) % 2 ? -1.0f : 1.0f;
        pc = fma(pc, x, df{sg * kInvFact[n][0], sg * kInvFact[n][1]});
    }
    const df cr = fma(pc, x, df{1.0f, 0.0f});
    const int q = (int)((long long)k & 3LL);
    const df s = (q & 1) ? cr : sr;
    const df c = (q & 1) ? sr : cr;
    return {(q & 2) ? neg(s) : s, ((q + 1) & 2) ? neg(c) : c};
}
// not inlined: the kernels that call it run it once or a few times per thread, and one copy of its
// ~300 instructions is fetched once per SM instead of at every call site
static __device__ __noinline__ df_sc df_sincos_nl(double th) { return df_sincos_v(th); }
__device__ __forceinline__ void df_sincos(double th, df* s_out, df* c_out) {
    const df_sc r = df_sincos_nl(th);
    *s_out = r.s;
    *c_out = r.c;
}

// ---- the same interface for double (FP64 mode)
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double shfl(double a, int src) { return __shfl_sync(0xffffffffu, a, src); }
__device__ __forceinline__ double shfl_up(double a, int off) { return __shfl_up_sync(0xffffffffu, a, off); }
__device__ __forceinline__ double shfl_down(double a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }

template <class T> __device__ __forceinline__ T num(double x);
template <> __device__ __forceinline__ double num<double>(double x) { return x; }
template <> __device__ __forceinline__ df num<df>(double x) { return df_from(x); }
template <class T> __device__ __forceinline__ T num_f(float x);
template <> __device__ __forceinline__ double num_f<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ df num_f<df>(float x) { return df{x, 0.0f}; }

}  // namespace dev
}  // namespace kcm
