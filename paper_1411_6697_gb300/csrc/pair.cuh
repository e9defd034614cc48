// pair.cuh -- device helpers for kernels that update two adjacent cells per
// thread: cp.async staging, exact conserved-moment sums and the recovery of
// rho, u, T (FP64 or double-float), and NND flux differences of a cell pair.
#pragma once
#include <float.h>

#include "cell.cuh"
#include "model.h"
#include "vec2.cuh"

namespace lbk {

__device__ __forceinline__ void cp16(void* dst, const void* src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// the hardware reciprocal approximation (about 1 ulp); every use refines it
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// the hardware square-root approximation (relative error about 2^-23), for the
// TNE measure d = sqrt(sum_k Delta_k^2), which is reported, never fed back
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct DfConst {
    float ch[4], cl[4], wh[4], wl[4], idh, idl, tigh, tigl;
};

// Conserved moments m1 = rho, m2 = rho u_x, m3 = rho u_y, m4 = rho[(D+I)T + u^2]
// (Eqs. (5)-(7)) of a pair of cells as double-float sums: every butterfly is an
// exact TwoSum, the orbit weights are applied as split constants.
__device__ __forceinline__ void conserved_pair(const V2* f, const DfConst& C, D2& m1, D2& m2,
                                               D2& m3, D2& m4)
{
    D2 P[2], E[2], AX[4], AY[4]; // sector slots: axis0, axis2 | diag1, diag3
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const int b = 8 * a;
        D2 s02 = two_sum(f[b], f[b + 2]), s13 = two_sum(f[b + 1], f[b + 3]);
        AX[a] = two_sum(f[b], -f[b + 2]);
        AY[a] = two_sum(f[b + 1], -f[b + 3]);
        P[a] = d_add(s02, s13);
    }
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const int b = 4 + 8 * d;
        D2 s01 = two_sum(f[b], f[b + 1]), d01 = two_sum(f[b], -f[b + 1]);
        D2 s23 = two_sum(f[b + 2], f[b + 3]), d23 = two_sum(f[b + 2], -f[b + 3]);
        E[d] = d_add(s01, s23);
        AY[2 + d] = d_add(s01, d_neg(s23));
        AX[2 + d] = d_add(d01, d_neg(d23));
    }
    // slot -> orbit: 0 -> 0, 1 -> 2, 2 -> 1, 3 -> 3
    m1 = d_add(d_add(P[0], P[1]), d_add(E[0], E[1]));
    m2 = d_add(d_add(d_mul_c(AX[0], C.ch[0], C.cl[0]), d_mul_c(AX[1], C.ch[2], C.cl[2])),
               d_add(d_mul_c(AX[2], C.ch[1], C.cl[1]), d_mul_c(AX[3], C.ch[3], C.cl[3])));
    m3 = d_add(d_add(d_mul_c(AY[0], C.ch[0], C.cl[0]), d_mul_c(AY[1], C.ch[2], C.cl[2])),
               d_add(d_mul_c(AY[2], C.ch[1], C.cl[1]), d_mul_c(AY[3], C.ch[3], C.cl[3])));
    m4 = d_add(d_add(d_mul_c(P[0], C.wh[0], C.wl[0]), d_mul_c(P[1], C.wh[2], C.wl[2])),
               d_add(d_mul_c(E[0], C.wh[1], C.wl[1]), d_mul_c(E[1], C.wh[3], C.wl[3])));
}

// The same conserved moments with the (hi, lo) pairs carried unnormalized through the
// butterflies: every hi + hi is an exact TwoSum (or TwoDiff), the lo parts and the
// rounding errors add in FP32 (each of size ulp(hi), so their own rounding is far below
// it), products with the split constants keep their error terms unnormalized, and each
// moment is normalized once at the end (FastTwoSum). Relative error about 2^-46.
__device__ __forceinline__ D2 two_diff(V2 a, V2 b)
{
    V2 s = a - b;
    V2 bb = s - a;
    V2 e = (a - (s - bb)) - (b + bb);
    return {s, e};
}
__device__ __forceinline__ D2 dd_add(D2 a, D2 b)
{
    const D2 s = two_sum(a.hi, b.hi);
    return {s.hi, (a.lo + b.lo) + s.lo};
}
__device__ __forceinline__ D2 dd_sub(D2 a, D2 b)
{
    const D2 s = two_diff(a.hi, b.hi);
    return {s.hi, (a.lo - b.lo) + s.lo};
}
__device__ __forceinline__ D2 dd_mul_c(D2 a, float ch, float cl)
{
    const V2 p = a.hi * ch;
    V2 e = fma(a.hi, V2(ch), -p);
    e = fma(a.hi, V2(cl), e);
    e = fma(a.lo, V2(ch), e);
    return {p, e};
}
__device__ __forceinline__ D2 dd_norm(D2 a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ void conserved_pair_u(const V2* f, const DfConst& C, D2& m1, D2& m2,
                                                 D2& m3, D2& m4)
{
    D2 P[2], E[2], AX[4], AY[4]; // sector slots: axis0, axis2 | diag1, diag3
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const int b = 8 * a;
        P[a] = dd_add(two_sum(f[b], f[b + 2]), two_sum(f[b + 1], f[b + 3]));
        AX[a] = two_diff(f[b], f[b + 2]);
        AY[a] = two_diff(f[b + 1], f[b + 3]);
    }
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const int b = 4 + 8 * d;
        const D2 s01 = two_sum(f[b], f[b + 1]), d01 = two_diff(f[b], f[b + 1]);
        const D2 s23 = two_sum(f[b + 2], f[b + 3]), d23 = two_diff(f[b + 2], f[b + 3]);
        E[d] = dd_add(s01, s23);
        AY[2 + d] = dd_sub(s01, s23);
        AX[2 + d] = dd_sub(d01, d23);
    }
    // slot -> orbit: 0 -> 0, 1 -> 2, 2 -> 1, 3 -> 3
    m1 = dd_norm(dd_add(dd_add(P[0], P[1]), dd_add(E[0], E[1])));
    m2 = dd_norm(dd_add(dd_add(dd_mul_c(AX[0], C.ch[0], C.cl[0]), dd_mul_c(AX[1], C.ch[2], C.cl[2])),
                        dd_add(dd_mul_c(AX[2], C.ch[1], C.cl[1]), dd_mul_c(AX[3], C.ch[3], C.cl[3]))));
    m3 = dd_norm(dd_add(dd_add(dd_mul_c(AY[0], C.ch[0], C.cl[0]), dd_mul_c(AY[1], C.ch[2], C.cl[2])),
                        dd_add(dd_mul_c(AY[2], C.ch[1], C.cl[1]), dd_mul_c(AY[3], C.ch[3], C.cl[3]))));
    m4 = dd_norm(dd_add(dd_add(dd_mul_c(P[0], C.wh[0], C.wl[0]), dd_mul_c(P[1], C.wh[2], C.wl[2])),
                        dd_add(dd_mul_c(E[0], C.wh[1], C.wl[1]), dd_mul_c(E[1], C.wh[3], C.wl[3]))));
}

// Double-float recovery: rho, u, T by corrected quotients on the FP32 pipes.
__device__ __forceinline__ void recover_pair_df(const V2* f, const DfConst& C, V2& rho, V2& ux,
                                                V2& uy, V2& T, bool& ig0, bool& ig1, bool& ok0,
                                                bool& ok1)
{
    D2 m1, m2, m3, m4;
    conserved_pair(f, C, m1, m2, m3, m4);
    const V2 rb(rcp_approx(m1.hi.x()), rcp_approx(m1.hi.y()));
    const D2 vx = d_div(m2, m1, rb), vy = d_div(m3, m1, rb), e = d_div(m4, m1, rb);
    const D2 t = d_mul_c(d_add(e, d_neg(d_add(d_sqr(vx), d_sqr(vy)))), C.idh, C.idl);
    rho = m1.hi;
    ux = vx.hi;
    uy = vy.hi;
    T = t.hi;
    ig0 = t.hi.x() > C.tigh || (t.hi.x() == C.tigh && t.lo.x() > C.tigl);
    ig1 = t.hi.y() > C.tigh || (t.hi.y() == C.tigh && t.lo.y() > C.tigl);
    ok0 = m1.hi.x() > 0.0f && t.hi.x() > 0.0f && t.hi.x() <= FLT_MAX;
    ok1 = m1.hi.y() > 0.0f && t.hi.y() > 0.0f && t.hi.y() <= FLT_MAX;
}

// Exact binary32 -> binary64 conversion by moving the IEEE-754 fields with integer
// operations (exponent rebias 127 -> 1023, significand shifted by 29 bits), so the
// conversion runs on the integer ALU instead of the FP64 unit, which GB300 builds
// for 1/58 of the FP32 rate. Zeros are built directly; subnormal, infinite and NaN
// inputs (never produced by a valid state) take the conversion instruction.
__device__ __forceinline__ double f2d_exact(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if (e - 1u < 254u) {
        const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
        return __hiloint2double((int)hi, (int)(b << 29));
    }
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)x;
}

// binary64 -> binary32, round to nearest even, by integer operations: the top 23
// significand bits are kept and the 29 dropped bits decide the rounding (above half:
// up; exactly half: to even). A carry out of the significand steps the exponent,
// which also yields infinity on overflow. Results outside the normal binary32 range
// (zero, subnormal) and infinite or NaN inputs take the conversion instruction.
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    if (e < 1 || e > 254) return __double2float_rn(x);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | (((unsigned)e << 23) + m + up));
}

// Ordered comparisons of FP64 values through their bit patterns: for a >= 0 (not
// NaN), x > a exactly when the patterns compare so as signed 64-bit integers.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// FP64 recovery: the exact conserved sums carried into FP64 (hi + lo), then rho,
// u, T formed in FP64 arithmetic.
// 1/m1 from an FP32 reciprocal refined by two FP64 Newton steps (each doubles the
// correct bits: 22 -> 44 -> full FP64), then u and T in FP64.
__device__ __forceinline__ void recover_one_f64(float seed_of, double m1, double m2, double m3,
                                                double m4, double inv_DI, double& u, double& v,
                                                double& t)
{
    double q = f2d_exact(rcp_approx(seed_of));
    q = ::fma(q, ::fma(-m1, q, 1.0), q);
    q = ::fma(q, ::fma(-m1, q, 1.0), q);
    u = m2 * q;
    v = m3 * q;
    t = (m4 * q - (u * u + v * v)) * inv_DI;
}

__device__ __forceinline__ double df_to_f64(float hi, float lo) { return f2d_exact(hi) + f2d_exact(lo); }

// rho, u, T of a cell pair from its 16 f: exact conserved sums, then FP64 (REC = 0)
// or double-float (REC = 1); ig = T > T_ig decided in that precision, ok = rho > 0
// and 0 < T < inf.
template <int REC>
__device__ __forceinline__ void recover_pair(const V2* f, const DfConst& C,
                                             const ModelConst<float>& K, V2& rho, V2& ux, V2& uy,
                                             V2& T, bool& ig0, bool& ig1, bool& ok0, bool& ok1)
{
    if constexpr (REC == 1) {
        recover_pair_df(f, C, rho, ux, uy, T, ig0, ig1, ok0, ok1);
    } else {
        D2 m1, m2, m3, m4;
        conserved_pair(f, C, m1, m2, m3, m4);
        double u0, v0, t0, u1, v1, t1;
        const double r0 = df_to_f64(m1.hi.x(), m1.lo.x());
        const double r1 = df_to_f64(m1.hi.y(), m1.lo.y());
        recover_one_f64(m1.hi.x(), r0, df_to_f64(m2.hi.x(), m2.lo.x()),
                        df_to_f64(m3.hi.x(), m3.lo.x()), df_to_f64(m4.hi.x(), m4.lo.x()),
                        K.inv_DId, u0, v0, t0);
        recover_one_f64(m1.hi.y(), r1, df_to_f64(m2.hi.y(), m2.lo.y()),
                        df_to_f64(m3.hi.y(), m3.lo.y()), df_to_f64(m4.hi.y(), m4.lo.y()),
                        K.inv_DId, u1, v1, t1);
        rho = m1.hi; // the exact sum rounded to FP32
        ux = V2(d2f_rn(u0), d2f_rn(u1));
        uy = V2(d2f_rn(v0), d2f_rn(v1));
        T = V2(d2f_rn(t0), d2f_rn(t1));
        const long long tig = dbits(K.T_igd), dmax = dbits(DBL_MAX);
        ig0 = dbits(t0) > tig;
        ig1 = dbits(t1) > tig;
        ok0 = dbits(r0) > 0 && dbits(t0) > 0 && dbits(t0) <= dmax;
        ok1 = dbits(r1) > 0 && dbits(t1) > 0 && dbits(t1) <= dmax;
    }
}

// Branch-free forms of the two conversions, for the values a step's recovery produces
// (normal binary32 / binary64 numbers of modest size, or zero):
// f2d_fast moves the IEEE-754 fields of a normal binary32 value into binary64 exactly
// (exponent rebias 127 -> 1023, significand shifted by 29 bits); a zero or subnormal
// input becomes +-2^-127 (below 6e-39), which added to a conserved sum of order one,
// or scaling a momentum that is exactly zero, changes nothing at FP32 output.
// d2f_fast rounds binary64 to binary32 to nearest even by adding the rounding bias to
// the 64-bit pattern (a carry steps the exponent), then shifting the top bits down and
// rebiasing the exponent; results below the normal binary32 range become a signed zero.
// Neither handles infinities or NaN: the recovery flags such cells from their FP32 sums
// before it converts anything.
__device__ __forceinline__ double f2d_fast(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned hi = (((b >> 3) & 0x0fffffffu) + (896u << 20)) | (b & 0x80000000u);
    return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ float d2f_fast(double x)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(bits >> 32);
    // round to nearest even at bit 29: + (2^28 - 1) + (bit 29)
    const unsigned long long r = bits + 0x0fffffffull + ((bits >> 29) & 1ull);
    const unsigned f = __funnelshift_r((unsigned)r, (unsigned)(r >> 32), 29) - (896u << 23);
    const bool normal = (hi & 0x7ff00000u) >= (897u << 20);
    return __uint_as_float(normal ? (f | (hi & 0x80000000u)) : (hi & 0x80000000u));
}
__device__ __forceinline__ double df_to_f64_fast(float hi, float lo) { return f2d_fast(hi) + f2d_fast(lo); }

// FP64 recovery of one cell with fewer FP64 operations: 1/m1 seeded by a double-float
// reciprocal formed on the FP32 pipes (the FP32 estimate r corrected by r (1 - m1 r),
// about 46 correct bits) and finished by one FP64 Newton step; u = m2 q, v = m3 q; and
// T = q (m4 - m2 u - m3 v) / (D+I), which equals (m4 q - u^2 - v^2) / (D+I).
__device__ __forceinline__ void recover_one_f64_fast(float m1h, float m1l, double m1, double m2,
                                                     double m3, double m4, double inv_DI,
                                                     double& u, double& v, double& t)
{
    const float r = rcp_approx(m1h);
    const float e = fmaf(-m1h, r, 1.0f) - m1l * r; // 1 - m1 r to FP32 accuracy
    double q = f2d_fast(r) + f2d_fast(r * e);
    q = ::fma(q, ::fma(-m1, q, 1.0), q);
    u = m2 * q;
    v = m3 * q;
    t = ::fma(-m3, v, ::fma(-m2, u, m4)) * (q * inv_DI);
}

// recover_pair with the branch-free conversions; cells whose conserved sums are not
// finite in FP32 are flagged before anything is converted.
template <int REC>
__device__ __forceinline__ void recover_pair_fast(const V2* f, const DfConst& C,
                                                  const ModelConst<float>& K, V2& rho, V2& ux,
                                                  V2& uy, V2& T, bool& ig0, bool& ig1, bool& ok0,
                                                  bool& ok1)
{
    if constexpr (REC == 1) {
        recover_pair_df(f, C, rho, ux, uy, T, ig0, ig1, ok0, ok1);
    } else {
        D2 m1, m2, m3, m4;
        conserved_pair_u(f, C, m1, m2, m3, m4);
        double u0, v0, t0, u1, v1, t1;
        const double r0 = df_to_f64_fast(m1.hi.x(), m1.lo.x());
        const double r1 = df_to_f64_fast(m1.hi.y(), m1.lo.y());
        recover_one_f64_fast(m1.hi.x(), m1.lo.x(), r0, df_to_f64_fast(m2.hi.x(), m2.lo.x()),
                             df_to_f64_fast(m3.hi.x(), m3.lo.x()), df_to_f64_fast(m4.hi.x(), m4.lo.x()),
                             K.inv_DId, u0, v0, t0);
        recover_one_f64_fast(m1.hi.y(), m1.lo.y(), r1, df_to_f64_fast(m2.hi.y(), m2.lo.y()),
                             df_to_f64_fast(m3.hi.y(), m3.lo.y()), df_to_f64_fast(m4.hi.y(), m4.lo.y()),
                             K.inv_DId, u1, v1, t1);
        rho = m1.hi; // the exact sum rounded to FP32
        ux = V2(d2f_fast(u0), d2f_fast(u1));
        uy = V2(d2f_fast(v0), d2f_fast(v1));
        T = V2(d2f_fast(t0), d2f_fast(t1));
        const long long tig = dbits(K.T_igd), dmax = dbits(DBL_MAX);
        ig0 = dbits(t0) > tig;
        ig1 = dbits(t1) > tig;
        const bool f0 = fabsf(m1.hi.x()) <= FLT_MAX && fabsf(m4.hi.x()) <= FLT_MAX;
        const bool f1 = fabsf(m1.hi.y()) <= FLT_MAX && fabsf(m4.hi.y()) <= FLT_MAX;
        ok0 = f0 && dbits(r0) > 0 && dbits(t0) > 0 && dbits(t0) <= dmax;
        ok1 = f1 && dbits(r1) > 0 && dbits(t1) > 0 && dbits(t1) <= dmax;
    }
}

// Split constants of the conserved-moment recovery (split on the host, so they stay
// constant-bank operands instead of registers).
__device__ __forceinline__ DfConst df_constants(const ModelConst<float>& K)
{
    DfConst C;
#pragma unroll
    for (int o = 0; o < 4; o++) {
        C.ch[o] = K.cdh[o];
        C.cl[o] = K.cdl[o];
        C.wh[o] = K.wdh[o];
        C.wl[o] = K.wdl[o];
    }
    C.idh = K.idh;
    C.idl = K.idl;
    C.tigh = K.tigh;
    C.tigl = K.tigl;
    return C;
}

// Plain FP32 velocity of one cell (halo columns, used only inside grad u).
__device__ __forceinline__ void velocity_f32(const float* f, const ModelConst<float>& K,
                                             float& ux, float& uy)
{
    float rho = 0.f;
#pragma unroll
    for (int i = 0; i < 16; i++) rho += f[i];
    const float jx = K.c[0] * (f[0] - f[2]) + K.c[2] * (f[8] - f[10]) +
                     K.c[1] * (f[4] - f[5] - f[6] + f[7]) + K.c[3] * (f[12] - f[13] - f[14] + f[15]);
    const float jy = K.c[0] * (f[1] - f[3]) + K.c[2] * (f[9] - f[11]) +
                     K.c[1] * (f[4] + f[5] - f[6] - f[7]) + K.c[3] * (f[12] + f[13] - f[14] - f[15]);
    ux = jx / rho;
    uy = jy / rho;
}

// NND flux differences of a pair of cells (x, x+1) along x, from q_{x-2..x+3}.
struct Q6 {
    float a, b, c, d, e, g; // x-2, x-1, x, x+1, x+2, x+3
};
__device__ __forceinline__ Q6 load6(const float* row, int lx)
{
    const float2 A = *reinterpret_cast<const float2*>(row + lx - 2);
    const float2 B = *reinterpret_cast<const float2*>(row + lx);
    const float2 Cc = *reinterpret_cast<const float2*>(row + lx + 2);
    return {A.x, A.y, B.x, B.y, Cc.x, Cc.y};
}
// |minmod(a, b)|: min(|a|, |b|) carrying sign(a) xor sign(b), then clamped at 0 (so 0
// unless a and b share a sign). Every nonzero minmod in an NND difference around the
// slope d has the sign of d, so mm(d, d') - mm(d'', d) = sign(d) (|mm(d, d')| -
// |mm(d'', d)|): the same value, rounded the same way.
__device__ __forceinline__ float mmag(float a, float b)
{
    float r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return fmaxf(r, 0.0f);
}
// x with its sign flipped where s is negative
__device__ __forceinline__ float sgnmul(float x, float s)
{
    return __uint_as_float(__float_as_uint(x) ^ (__float_as_uint(s) & 0x80000000u));
}
__device__ __forceinline__ V2 sgnmul(V2 x, V2 s) { return V2(sgnmul(x.x(), s.x()), sgnmul(x.y(), s.y())); }
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// upwind side v > 0: (d1 + (mm(d1,d2) - mm(d0,d1))/2) for both cells
__device__ __forceinline__ V2 nnd_pos_x(const Q6& q)
{
    const float d0 = q.b - q.a, d1 = q.c - q.b, d2 = q.d - q.c, d3 = q.e - q.d;
    const float r01 = mmag(d0, d1), r12 = mmag(d1, d2), r23 = mmag(d2, d3);
    const V2 s(d1, d2);
    return fma(V2(0.5f), sgnmul(V2(r12, r23) - V2(r01, r12), s), s);
}
// upwind side v < 0: (d2 - (mm(d2,d3) - mm(d1,d2))/2) for both cells
__device__ __forceinline__ V2 nnd_neg_x(const Q6& q)
{
    const float d1 = q.c - q.b, d2 = q.d - q.c, d3 = q.e - q.d, d4 = q.g - q.e;
    const float r12 = mmag(d1, d2), r23 = mmag(d2, d3), r34 = mmag(d3, d4);
    const V2 s(d2, d3);
    return fma(V2(-0.5f), sgnmul(V2(r23, r34) - V2(r12, r23), s), s);
}
__device__ __forceinline__ V2 ldv(const float* p) { return V2(*reinterpret_cast<const float2*>(p)); }
// along y from rows y-2..y+1 (v > 0) or y-1..y+2 (v < 0), packed over the pair
__device__ __forceinline__ V2 nnd_pos_y(V2 qm2, V2 qm1, V2 q0, V2 qp1)
{
    const V2 d0 = qm1 - qm2, d1 = q0 - qm1, d2 = qp1 - q0;
    const V2 r12(mmag(d1.x(), d2.x()), mmag(d1.y(), d2.y()));
    const V2 r01(mmag(d0.x(), d1.x()), mmag(d0.y(), d1.y()));
    return fma(V2(0.5f), sgnmul(r12 - r01, d1), d1);
}
__device__ __forceinline__ V2 nnd_neg_y(V2 qm1, V2 q0, V2 qp1, V2 qp2)
{
    const V2 d1 = q0 - qm1, d2 = qp1 - q0, d3 = qp2 - qp1;
    const V2 r23(mmag(d2.x(), d3.x()), mmag(d2.y(), d3.y()));
    const V2 r12(mmag(d1.x(), d2.x()), mmag(d1.y(), d2.y()));
    return fma(V2(-0.5f), sgnmul(r23 - r12, d2), d2);
}

} // namespace lbk
