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

struct DfConst {
    float ch[4], cl[4], wh[4], wl[4], idh, idl, tigh, tigl;
};

__device__ __forceinline__ void split(double v, float& h, float& l)
{
    h = (float)v;
    l = (float)(v - (double)h);
}

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

// Double-float recovery: rho, u, T by corrected quotients on the FP32 pipes.
__device__ __forceinline__ void recover_pair_df(const V2* f, const DfConst& C, V2& rho, V2& ux,
                                                V2& uy, V2& T, bool& ig0, bool& ig1, bool& ok0,
                                                bool& ok1)
{
    D2 m1, m2, m3, m4;
    conserved_pair(f, C, m1, m2, m3, m4);
    const V2 rb(__frcp_rn(m1.hi.x()), __frcp_rn(m1.hi.y()));
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

// FP64 recovery: the exact conserved sums carried into FP64 (hi + lo), then rho,
// u, T formed in FP64 arithmetic.
// 1/m1 from an FP32 reciprocal refined by two FP64 Newton steps (each doubles the
// correct bits: 24 -> 48 -> full FP64), then u and T in FP64.
__device__ __forceinline__ void recover_one_f64(float seed_of, double m1, double m2, double m3,
                                                double m4, double inv_DI, double& u, double& v,
                                                double& t)
{
    double q = (double)__frcp_rn(seed_of);
    q = ::fma(q, ::fma(-m1, q, 1.0), q);
    q = ::fma(q, ::fma(-m1, q, 1.0), q);
    u = m2 * q;
    v = m3 * q;
    t = (m4 * q - (u * u + v * v)) * inv_DI;
}

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
        const double r0 = (double)m1.hi.x() + (double)m1.lo.x();
        const double r1 = (double)m1.hi.y() + (double)m1.lo.y();
        recover_one_f64(m1.hi.x(), r0, (double)m2.hi.x() + (double)m2.lo.x(),
                        (double)m3.hi.x() + (double)m3.lo.x(), (double)m4.hi.x() + (double)m4.lo.x(),
                        K.inv_DId, u0, v0, t0);
        recover_one_f64(m1.hi.y(), r1, (double)m2.hi.y() + (double)m2.lo.y(),
                        (double)m3.hi.y() + (double)m3.lo.y(), (double)m4.hi.y() + (double)m4.lo.y(),
                        K.inv_DId, u1, v1, t1);
        rho = m1.hi; // the exact sum rounded to FP32
        ux = V2((float)u0, (float)u1);
        uy = V2((float)v0, (float)v1);
        T = V2((float)t0, (float)t1);
        ig0 = t0 > K.T_igd;
        ig1 = t1 > K.T_igd;
        ok0 = r0 > 0.0 && t0 > 0.0 && t0 <= DBL_MAX;
        ok1 = r1 > 0.0 && t1 > 0.0 && t1 <= DBL_MAX;
    }
}

// Split constants of the conserved-moment recovery, from the FP64 model constants.
__device__ __forceinline__ DfConst df_constants(const ModelConst<float>& K)
{
    DfConst C;
#pragma unroll
    for (int o = 0; o < 4; o++) {
        split(K.cd[o], C.ch[o], C.cl[o]);
        split(K.wd[o], C.wh[o], C.wl[o]);
    }
    split(K.inv_DId, C.idh, C.idl);
    split(K.T_igd, C.tigh, C.tigl);
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
// upwind side v > 0: (d1 + (mm(d1,d2) - mm(d0,d1))/2) for both cells
__device__ __forceinline__ V2 nnd_pos_x(const Q6& q)
{
    const float d0 = q.b - q.a, d1 = q.c - q.b, d2 = q.d - q.c, d3 = q.e - q.d;
    const float m01 = mm1(d0, d1), m12 = mm1(d1, d2), m23 = mm1(d2, d3);
    return fma(V2(0.5f), V2(m12, m23) - V2(m01, m12), V2(d1, d2));
}
// upwind side v < 0: (d2 - (mm(d2,d3) - mm(d1,d2))/2) for both cells
__device__ __forceinline__ V2 nnd_neg_x(const Q6& q)
{
    const float d1 = q.c - q.b, d2 = q.d - q.c, d3 = q.e - q.d, d4 = q.g - q.e;
    const float m12 = mm1(d1, d2), m23 = mm1(d2, d3), m34 = mm1(d3, d4);
    return fma(V2(-0.5f), V2(m23, m34) - V2(m12, m23), V2(d2, d3));
}
__device__ __forceinline__ V2 ldv(const float* p) { return V2(*reinterpret_cast<const float2*>(p)); }
// along y from rows y-2..y+1 (v > 0) or y-1..y+2 (v < 0), packed over the pair
__device__ __forceinline__ V2 nnd_pos_y(V2 qm2, V2 qm1, V2 q0, V2 qp1)
{
    const V2 d0 = qm1 - qm2, d1 = q0 - qm1, d2 = qp1 - q0;
    return fma(V2(0.5f), mm2(d1, d2) - mm2(d0, d1), d1);
}
__device__ __forceinline__ V2 nnd_neg_y(V2 qm1, V2 q0, V2 qp1, V2 qp2)
{
    const V2 d1 = q0 - qm1, d2 = qp1 - q0, d3 = qp2 - qp1;
    return fma(V2(-0.5f), mm2(d2, d3) - mm2(d1, d2), d2);
}

} // namespace lbk
