// vec2.cuh -- two cells per thread with the packed FP32 instructions of sm_100+
// (FFMA2 / FADD2 / FMUL2 via __ffma2_rn, __fadd2_rn, __fmul2_rn), and
// double-float arithmetic on such pairs (error-free transforms).
#pragma once
#include <cuda_runtime.h>

namespace lbk {

struct V2 {
    float2 v;
    __device__ __forceinline__ V2() {}
    __device__ __forceinline__ V2(float2 a) : v(a) {}
    // lane c of the pair (c a compile-time constant after unrolling)
    __device__ __forceinline__ float operator[](int c) const { return c ? v.y : v.x; }
    __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit V2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
};

__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator*(float a, V2 b) { return V2(__fmul2_rn(make_float2(a, a), b.v)); }
__device__ __forceinline__ V2 operator*(V2 a, float b) { return V2(__fmul2_rn(a.v, make_float2(b, b))); }
// a - b as one packed FMA: b * (-1) + a (exact product, one rounding)
__device__ __forceinline__ V2 operator-(V2 a, V2 b)
{
    return V2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ V2 operator-(V2 a) { return V2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 operator+(V2 a, float b) { return a + V2(b); }
__device__ __forceinline__ V2 operator-(V2 a, float b) { return a - V2(b); }
__device__ __forceinline__ V2 operator+(float a, V2 b) { return V2(a) + b; }
__device__ __forceinline__ V2 operator-(float a, V2 b) { return V2(a) - b; }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) { return a = a + b; }
__device__ __forceinline__ V2 fma(V2 a, V2 b, V2 c) { return V2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ V2 fma(float a, V2 b, V2 c)
{
    return V2(__ffma2_rn(make_float2(a, a), b.v, c.v));
}
__device__ __forceinline__ V2 vmin(V2 a, V2 b) { return V2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ V2 vmax(V2 a, V2 b) { return V2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
__device__ __forceinline__ V2 lane_recip(V2 a) { return V2(1.0f / a.v.x, 1.0f / a.v.y); }
__device__ __forceinline__ V2 vabs(V2 a) { return V2(fabsf(a.v.x), fabsf(a.v.y)); }

// minmod(a, b) is the median of a, b and 0: four min/max operations, no arithmetic
__device__ __forceinline__ float mm1(float a, float b)
{
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}
__device__ __forceinline__ V2 mm2(V2 a, V2 b) { return V2(mm1(a.v.x, b.v.x), mm1(a.v.y, b.v.y)); }

// ---- double-float pairs (hi + lo, |lo| <= ulp(hi)/2 after normalisation) ----
struct D2 {
    V2 hi, lo;
};
// s + e == a + b exactly (Knuth)
__device__ __forceinline__ D2 two_sum(V2 a, V2 b)
{
    V2 s = a + b;
    V2 bb = s - a;
    V2 e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// s + e == a + b exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ D2 fast_two_sum(V2 a, V2 b)
{
    V2 s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ D2 d_add(D2 a, D2 b)
{
    D2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ D2 d_neg(D2 a) { return {-a.hi, -a.lo}; }
// a * (ch + cl) for a double constant split into two floats
__device__ __forceinline__ D2 d_mul_c(D2 a, float ch, float cl)
{
    V2 p = a.hi * ch;
    V2 e = fma(a.hi, V2(ch), -p);
    e = fma(a.hi, V2(cl), e);
    e = fma(a.lo, V2(ch), e);
    return fast_two_sum(p, e);
}
// a / b with one correction of the FP32 quotient
__device__ __forceinline__ D2 d_div(D2 a, D2 b, V2 rb)
{
    V2 q = a.hi * rb;
    V2 r = fma(-b.hi, q, a.hi);  // exact remainder of the hi parts up to b.lo
    r = r + (a.lo - b.lo * q);
    return fast_two_sum(q, r * rb);
}
__device__ __forceinline__ D2 d_sqr(D2 a)
{
    V2 p = a.hi * a.hi;
    V2 e = fma(a.hi, a.hi, -p);
    e = fma(V2(2.0f) * a.hi, a.lo, e);
    return fast_two_sum(p, e);
}

} // namespace lbk
