// Double-float arithmetic: a value held as the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
//
// On this GPU the FP64 fused multiply-add issues at under two lanes per
// clock per SM against 128 for FP32, so a double-float operation of 6 to 11
// FP32 instructions runs several times faster than one FP64 instruction.
// The borderline re-pass of the integrator (right-hand side of Eq. 1 at a
// relative accuracy far below its tolerance 1e-9) uses it in place of FP64.
//
// The building blocks are the error-free transformations of Knuth (two-sum)
// and Dekker (fast two-sum, |a| >= |b|) and the FMA-based exact product;
// the operations follow the double-double algorithms of Hida, Li and Bailey
// ("sloppy" addition: the error is relative to |a| + |b|, not to the sum).
// Every FP32 step is an explicit round-to-nearest intrinsic, which the
// compiler never contracts or reassociates.  Exponent range is FP32's:
// callers keep magnitudes within about 2^+-120.
#pragma once

namespace grins {

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dd(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ constexpr dd(int i) : hi((float)i), lo(0.0f) {}            // |i| < 2^24: exact
    __host__ __device__ constexpr dd(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi; }
};

// s + e with |s| >= |e| (or s = 0) as a normalised pair
__device__ __forceinline__ dd dd_fast2(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return dd(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dd operator+(dd a, dd b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return dd_fast2(s, e);
}

__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dd_fast2(p, e);
}

// a * f for an FP32 f
__device__ __forceinline__ dd dd_mulf(dd a, float f)
{
    const float p = __fmul_rn(a.hi, f);
    float e = __fmaf_rn(a.hi, f, -p);
    e = __fmaf_rn(a.lo, f, e);
    return dd_fast2(p, e);
}

// a / b: a quotient from the approximate reciprocal of b.hi, corrected once
// by the remainder a - q b (relative error about 2^-44)
__device__ __forceinline__ dd operator/(dd a, dd b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b.hi));
    const float q1 = __fmul_rn(a.hi, r);
    const dd rem = a - dd_mulf(b, q1);
    const float q2 = __fmul_rn(rem.hi, r);
    return dd_fast2(q1, q2);
}

__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
__device__ __forceinline__ dd &operator*=(dd &a, dd b) { return a = a * b; }

__device__ __forceinline__ bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dd a, dd b) { return b < a; }
__device__ __forceinline__ bool operator<=(dd a, dd b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
__device__ __forceinline__ bool operator>=(dd a, dd b) { return b <= a; }

// finite: neither part has the all-ones exponent of an infinity or a NaN
__device__ __forceinline__ bool dd_isfinite(dd a)
{
    return (__float_as_int(a.hi) & 0x7f800000) != 0x7f800000 && (__float_as_int(a.lo) & 0x7f800000) != 0x7f800000;
}
__device__ __forceinline__ dd dd_abs(dd a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ dd dd_max(dd a, dd b) { return a < b ? b : a; }
__device__ __forceinline__ dd dd_min(dd a, dd b) { return b < a ? b : a; }

// a * 2^k for an integer k with 2^k a normal FP32 number: exact
__device__ __forceinline__ dd dd_ldexp(dd a, int k)
{
    const float s = __int_as_float((127 + k) << 23);
    return dd(__fmul_rn(a.hi, s), __fmul_rn(a.lo, s));
}

// Binary exponent of a normal positive FP32 number
__device__ __forceinline__ int dd_expo(float x) { return ((__float_as_int(x) >> 23) & 0xff) - 127; }

__device__ __forceinline__ dd dd_shfl_xor(dd v, int o)
{
    return dd(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace grins
