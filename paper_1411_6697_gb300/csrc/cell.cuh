// cell.cuh -- per-cell arithmetic of one MRT-LBKM step (device side).
//
// Block-form moment transforms (see model.h), conserved-moment recovery,
// equilibrium moments and their T-derivative, the NND flux difference and the
// reaction increment. Templated on the arithmetic type R (float or double).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "model.h"

namespace lbk {

template <typename R>
__device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }
template <typename R>
__device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }

// minmod of the NND scheme: 0 unless a and b share a sign, else the one of
// smaller magnitude -- which is the median of a, b and 0, written as
// max(min(a,b), min(max(a,b),0)).
template <typename R>
__device__ __forceinline__ R minmod(R a, R b)
{
    return rmax(rmin(a, b), rmin(rmax(a, b), R(0)));
}

// (H_{j+1/2} - H_{j-1/2}) / v of the NND flux of F = v q for v > 0, from
// q_{j-2}, q_{j-1}, q_j, q_{j+1}: the interface value is q_j + mm(dq_j, dq_{j+1})/2.
template <typename R>
__device__ __forceinline__ R nnd_pos(R qm2, R qm1, R q0, R qp1)
{
    R d0 = qm1 - qm2, d1 = q0 - qm1, d2 = qp1 - q0;
    return d1 + R(0.5) * (minmod(d1, d2) - minmod(d0, d1));
}

// the same for v < 0 from q_{j-1}, q_j, q_{j+1}, q_{j+2}: the interface value
// is q_{j+1} - mm(dq_{j+1}, dq_{j+2})/2.
template <typename R>
__device__ __forceinline__ R nnd_neg(R qm1, R q0, R qp1, R qp2)
{
    R d1 = q0 - qm1, d2 = qp1 - q0, d3 = qp2 - qp1;
    return d2 - R(0.5) * (minmod(d2, d3) - minmod(d1, d2));
}

// y = A x for an N x N block A of coefficients (type T) acting on lanes of type L
// (a scalar, or a pair of cells packed for FFMA2).
template <int N, typename T, typename L>
__device__ __forceinline__ void matvec(const T* A, const L* x, L* y)
{
#pragma unroll
    for (int r = 0; r < N; r++) {
        L s = A[r * N] * x[0];
#pragma unroll
        for (int c = 1; c < N; c++) s = fma(A[r * N + c], x[c], s);
        y[r] = s;
    }
}

// f (velocity space, orbit-major) -> the 16 moments in the standard order
// m1..m16 (0-based index k-1), by butterflies and the sector blocks.
template <typename R, typename L>
__device__ __forceinline__ void forward_moments(const ModelConst<R>& K, const L* f, L* m)
{
    // axis orbits 0 (f0..f3) and 2 (f8..f11)
    L sx0 = f[0] + f[2], sy0 = f[1] + f[3], ax0 = f[0] - f[2], ay0 = f[1] - f[3];
    L sx2 = f[8] + f[10], sy2 = f[9] + f[11], ax2 = f[8] - f[10], ay2 = f[9] - f[11];
    // diagonal orbits 1 (f4..f7) and 3 (f12..f15)
    L s01 = f[4] + f[5], d01 = f[4] - f[5], s23 = f[6] + f[7], d23 = f[6] - f[7];
    L e1 = s01 + s23, ay1 = s01 - s23, ax1 = d01 - d23, o1 = d01 + d23;
    L t01 = f[12] + f[13], u01 = f[12] - f[13], t23 = f[14] + f[15], u23 = f[14] - f[15];
    L e3 = t01 + t23, ay3 = t01 - t23, ax3 = u01 - u23, o3 = u01 + u23;

    L es[4] = {sx0 + sy0, sx2 + sy2, e1, e3}, ea[2] = {sx0 - sy0, sx2 - sy2};
    L xo[4] = {ax0, ax2, ax1, ax3}, yo[4] = {ay0, ay2, ay1, ay3}, oo[2] = {o1, o3};
    L pes[4], pea[2], px[4], py[4], po[2];
    matvec<4>(K.Bes, es, pes);
    matvec<2>(K.Bea, ea, pea);
    matvec<4>(K.Bodd, xo, px);
    matvec<4>(K.Bodd, yo, py);
    matvec<2>(K.Boo, oo, po);
    m[0] = pes[0];
    m[3] = pes[1];
    m[4] = L(0.5f) * (pes[2] + pea[0]);
    m[6] = L(0.5f) * (pes[2] - pea[0]);
    m[13] = L(0.5f) * (pes[3] + pea[1]);
    m[15] = L(0.5f) * (pes[3] - pea[1]);
    m[1] = px[0];
    m[7] = px[1];
    m[9] = px[2];
    m[11] = px[3];
    m[2] = py[0];
    m[8] = py[1];
    m[12] = py[2];
    m[10] = py[3];
    m[5] = po[0];
    m[14] = po[1];
}

// moments (standard order) -> velocity space: Omega = M^-1 Omega_hat.
template <typename R, typename L>
__device__ __forceinline__ void inverse_moments(const ModelConst<R>& K, const L* mh, L* f)
{
    L es[4] = {mh[0], mh[3], mh[4] + mh[6], mh[13] + mh[15]};
    L ea[2] = {mh[4] - mh[6], mh[13] - mh[15]};
    L xo[4] = {mh[1], mh[7], mh[9], mh[11]};
    L yo[4] = {mh[2], mh[8], mh[12], mh[10]};
    L oo[2] = {mh[5], mh[14]};
    L pes[4], pea[2], px[4], py[4], po[2];
    matvec<4>(K.Ies, es, pes);
    matvec<2>(K.Iea, ea, pea);
    matvec<4>(K.Iodd, xo, px);
    matvec<4>(K.Iodd, yo, py);
    matvec<2>(K.Ioo, oo, po);
    // axis orbits
#pragma unroll
    for (int a = 0; a < 2; a++) {
        L pp = pes[a] + pea[a], pm = pes[a] - pea[a];
        f[8 * a + 0] = pp + px[a];
        f[8 * a + 2] = pp - px[a];
        f[8 * a + 1] = pm + py[a];
        f[8 * a + 3] = pm - py[a];
    }
    // diagonal orbits
#pragma unroll
    for (int d = 0; d < 2; d++) {
        L e = pes[2 + d], X = px[2 + d], Y = py[2 + d], o = po[d];
        L eo = e + o, em = e - o, xp = X + Y, xm = X - Y;
        f[4 + 8 * d + 0] = eo + xp;
        f[4 + 8 * d + 1] = em - xm;
        f[4 + 8 * d + 2] = eo - xp;
        f[4 + 8 * d + 3] = em + xm;
    }
}

// y = A^T x for an N x N block A (the transpose of matvec)
template <int N, typename T, typename L>
__device__ __forceinline__ void matvec_t(const T* A, const L* x, L* y)
{
#pragma unroll
    for (int c = 0; c < N; c++) {
        L s = A[c] * x[0];
#pragma unroll
        for (int r = 1; r < N; r++) s = fma(A[r * N + c], x[r], s);
        y[c] = s;
    }
}

// fb = M^T mb: the transpose of forward_moments, its steps reversed (moment placement,
// sector blocks, the sector sums, the orbit butterflies), for the adjoint.
template <typename R, typename L>
__device__ __forceinline__ void forward_moments_t(const ModelConst<R>& K, const L* mb, L* fb)
{
    L pes[4] = {mb[0], mb[3], L(0.5) * (mb[4] + mb[6]), L(0.5) * (mb[13] + mb[15])};
    L pea[2] = {L(0.5) * (mb[4] - mb[6]), L(0.5) * (mb[13] - mb[15])};
    L px[4] = {mb[1], mb[7], mb[9], mb[11]}, py[4] = {mb[2], mb[8], mb[12], mb[10]};
    L po[2] = {mb[5], mb[14]};
    L es[4], ea[2], xo[4], yo[4], oo[2];
    matvec_t<4>(K.Bes, pes, es);
    matvec_t<2>(K.Bea, pea, ea);
    matvec_t<4>(K.Bodd, px, xo);
    matvec_t<4>(K.Bodd, py, yo);
    matvec_t<2>(K.Boo, po, oo);
    // axis orbits 0 (f0..f3) and 2 (f8..f11): es[a] = sx + sy, ea[a] = sx - sy
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const L sx = es[a] + ea[a], sy = es[a] - ea[a];
        fb[8 * a + 0] = sx + xo[a];
        fb[8 * a + 2] = sx - xo[a];
        fb[8 * a + 1] = sy + yo[a];
        fb[8 * a + 3] = sy - yo[a];
    }
    // diagonal orbits 1 (f4..f7) and 3 (f12..f15): e = s01 + s23, a_y = s01 - s23,
    // a_x = d01 - d23, o = d01 + d23
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const L e = es[2 + d], ax = xo[2 + d], ay = yo[2 + d], o = oo[d];
        const L s01 = e + ay, s23 = e - ay, d01 = ax + o, d23 = o - ax;
        fb[4 + 8 * d + 0] = s01 + d01;
        fb[4 + 8 * d + 1] = s01 - d01;
        fb[4 + 8 * d + 2] = s23 + d23;
        fb[4 + 8 * d + 3] = s23 - d23;
    }
}

// mb = M^-T fb: the transpose of inverse_moments, its steps reversed, for the adjoint.
template <typename R, typename L>
__device__ __forceinline__ void inverse_moments_t(const ModelConst<R>& K, const L* fb, L* mb)
{
    L pes[4], pea[2], px[4], py[4], po[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const L pp = fb[8 * a + 0] + fb[8 * a + 2], pm = fb[8 * a + 1] + fb[8 * a + 3];
        px[a] = fb[8 * a + 0] - fb[8 * a + 2];
        py[a] = fb[8 * a + 1] - fb[8 * a + 3];
        pes[a] = pp + pm;
        pea[a] = pp - pm;
    }
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const L f0 = fb[4 + 8 * d + 0], f1 = fb[4 + 8 * d + 1];
        const L f2 = fb[4 + 8 * d + 2], f3 = fb[4 + 8 * d + 3];
        const L eo = f0 + f2, xp = f0 - f2, em = f1 + f3, xm = f3 - f1;
        pes[2 + d] = eo + em;
        po[d] = eo - em;
        px[2 + d] = xp + xm;
        py[2 + d] = xp - xm;
    }
    L es[4], ea[2], xo[4], yo[4], oo[2];
    matvec_t<4>(K.Ies, pes, es);
    matvec_t<2>(K.Iea, pea, ea);
    matvec_t<4>(K.Iodd, px, xo);
    matvec_t<4>(K.Iodd, py, yo);
    matvec_t<2>(K.Ioo, po, oo);
    mb[0] = es[0];
    mb[3] = es[1];
    mb[4] = es[2] + ea[0];
    mb[6] = es[2] - ea[0];
    mb[13] = es[3] + ea[1];
    mb[15] = es[3] - ea[1];
    mb[1] = xo[0];
    mb[7] = xo[1];
    mb[9] = xo[2];
    mb[11] = xo[3];
    mb[2] = yo[0];
    mb[8] = yo[1];
    mb[12] = yo[2];
    mb[10] = yo[3];
    mb[5] = oo[0];
    mb[14] = oo[1];
}

// Conserved moments rho, rho u, rho[(D+I)T + u^2] (Eqs. (5)-(7)) from the 16 f
// in FP64, and rho, u, T from them, also in FP64.
template <typename F>
__device__ __forceinline__ void recover_f64(const double* cd, const double* wd, double inv_DI,
                                            const F* fin, double& rho, double& ux, double& uy,
                                            double& T)
{
    double f[16];
#pragma unroll
    for (int i = 0; i < 16; i++) f[i] = (double)fin[i];
    double sx0 = f[0] + f[2], sy0 = f[1] + f[3], ax0 = f[0] - f[2], ay0 = f[1] - f[3];
    double sx2 = f[8] + f[10], sy2 = f[9] + f[11], ax2 = f[8] - f[10], ay2 = f[9] - f[11];
    double s01 = f[4] + f[5], d01 = f[4] - f[5], s23 = f[6] + f[7], d23 = f[6] - f[7];
    double t01 = f[12] + f[13], u01 = f[12] - f[13], t23 = f[14] + f[15], u23 = f[14] - f[15];
    double P0 = sx0 + sy0, P2 = sx2 + sy2, e1 = s01 + s23, e3 = t01 + t23;
    double m1 = (P0 + P2) + (e1 + e3);
    double m2 = cd[0] * ax0 + cd[2] * ax2 + cd[1] * (d01 - d23) + cd[3] * (u01 - u23);
    double m3 = cd[0] * ay0 + cd[2] * ay2 + cd[1] * (s01 - s23) + cd[3] * (t01 - t23);
    double m4 = wd[0] * P0 + wd[2] * P2 + wd[1] * e1 + wd[3] * e3;
    double r = 1.0 / m1;
    rho = m1;
    ux = m2 * r;
    uy = m3 * r;
    T = (m4 * r - (ux * ux + uy * uy)) * inv_DI;
}

// ---- double-float (pairs of FP32) recovery ------------------------------
// Error-free transforms (Knuth TwoSum, FMA-based TwoProd) give each conserved
// moment as hi + lo with ~48 significant bits, on the FP32 pipes.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return two_sum(p, e);
}
__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return two_sum(p, e);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }
// a / b by one Newton correction of the FP32 quotient
__device__ __forceinline__ df df_div(df a, df b)
{
    float q1 = a.hi / b.hi;
    df r = df_sub(a, df_mul_f(b, q1));
    float q2 = r.hi / b.hi;
    r = df_sub(r, df_mul_f(b, q2));
    float q3 = r.hi / b.hi;
    df q = two_sum(q1, q2);
    return df_add(q, {q3, 0.0f});
}
// constant c given as a double split into hi + lo floats
__device__ __forceinline__ df df_const(double c)
{
    float h = (float)c;
    return {h, (float)(c - (double)h)};
}

__device__ __forceinline__ void recover_df32(const double* cd, const double* wd, double inv_DI,
                                             const float* f, double& rho, double& ux, double& uy,
                                             double& T)
{
    // butterflies with exact error terms
    df sx0 = two_sum(f[0], f[2]), sy0 = two_sum(f[1], f[3]);
    df ax0 = two_sum(f[0], -f[2]), ay0 = two_sum(f[1], -f[3]);
    df sx2 = two_sum(f[8], f[10]), sy2 = two_sum(f[9], f[11]);
    df ax2 = two_sum(f[8], -f[10]), ay2 = two_sum(f[9], -f[11]);
    df s01 = two_sum(f[4], f[5]), d01 = two_sum(f[4], -f[5]);
    df s23 = two_sum(f[6], f[7]), d23 = two_sum(f[6], -f[7]);
    df t01 = two_sum(f[12], f[13]), u01 = two_sum(f[12], -f[13]);
    df t23 = two_sum(f[14], f[15]), u23 = two_sum(f[14], -f[15]);
    df P0 = df_add(sx0, sy0), P2 = df_add(sx2, sy2);
    df e1 = df_add(s01, s23), e3 = df_add(t01, t23);
    df m1 = df_add(df_add(P0, P2), df_add(e1, e3));
    df ax1 = df_sub(d01, d23), ax3 = df_sub(u01, u23);
    df ay1 = df_sub(s01, s23), ay3 = df_sub(t01, t23);
    df c0 = df_const(cd[0]), c1 = df_const(cd[1]), c2 = df_const(cd[2]), c3 = df_const(cd[3]);
    df m2 = df_add(df_add(df_mul(ax0, c0), df_mul(ax2, c2)),
                   df_add(df_mul(ax1, c1), df_mul(ax3, c3)));
    df m3 = df_add(df_add(df_mul(ay0, c0), df_mul(ay2, c2)),
                   df_add(df_mul(ay1, c1), df_mul(ay3, c3)));
    df w0 = df_const(wd[0]), w1 = df_const(wd[1]), w2 = df_const(wd[2]), w3 = df_const(wd[3]);
    df m4 = df_add(df_add(df_mul(P0, w0), df_mul(P2, w2)), df_add(df_mul(e1, w1), df_mul(e3, w3)));
    df vx = df_div(m2, m1), vy = df_div(m3, m1);
    df e = df_div(m4, m1);
    df u2 = df_add(df_mul(vx, vx), df_mul(vy, vy));
    df t = df_mul(df_sub(e, u2), df_const(inv_DI));
    rho = (double)m1.hi + (double)m1.lo;
    ux = (double)vx.hi + (double)vx.lo;
    uy = (double)vy.hi + (double)vy.lo;
    T = (double)t.hi + (double)t.lo;
}

// Equilibrium moments f_hat^eq_1..16 (Sec. II; entries 14 and 16 per Eq. (11)).
template <typename R>
__device__ __forceinline__ void feq_moments(R DI, R rho, R ux, R uy, R T, R* q)
{
    R u2 = ux * ux + uy * uy;
    R A = (DI + R(2)) * T + u2;
    R B = (DI + R(4)) * T + u2;
    R rux = rho * ux, ruy = rho * uy;
    q[0] = rho;
    q[1] = rux;
    q[2] = ruy;
    q[3] = rho * (DI * T + u2);
    q[4] = rho * (T + ux * ux);
    q[5] = rux * uy;
    q[6] = rho * (T + uy * uy);
    q[7] = rux * A;
    q[8] = ruy * A;
    q[9] = rux * (R(3) * T + ux * ux);
    q[10] = ruy * (T + ux * ux);
    q[11] = rux * (T + uy * uy);
    q[12] = ruy * (R(3) * T + uy * uy);
    q[13] = rho * A * T + rux * ux * B;
    q[14] = rux * uy * B;
    q[15] = rho * A * T + ruy * uy * B;
}

// d f_hat^eq_k / dT at fixed rho, u (chemical term, Eqs. (19)-(23)).
template <typename R>
__device__ __forceinline__ void dfeq_dT(R DI, R rho, R ux, R uy, R T, R* d)
{
    R u2 = ux * ux + uy * uy;
    R dAT = R(2) * (DI + R(2)) * T + u2;
    R rux = rho * ux, ruy = rho * uy;
    d[0] = d[1] = d[2] = R(0);
    d[3] = rho * DI;
    d[4] = rho;
    d[5] = R(0);
    d[6] = rho;
    d[7] = rux * (DI + R(2));
    d[8] = ruy * (DI + R(2));
    d[9] = R(3) * rux;
    d[10] = ruy;
    d[11] = rux;
    d[12] = R(3) * ruy;
    d[13] = rho * dAT + rux * ux * (DI + R(4));
    d[14] = rux * uy * (DI + R(4));
    d[15] = rho * dAT + ruy * uy * (DI + R(4));
}

__device__ __forceinline__ float expm1_r(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_r(double x) { return expm1(x); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

// Exact increment of lambda over dt from d(lambda)/dt = (1-lambda)(a + b lambda),
// a = omega1 p, b = omega2 p (Eq. (28), m = n = 1).
template <typename R>
__device__ __forceinline__ R reaction_increment(R lam, R a, R b, R dt)
{
    R mu0 = R(1) - lam;
    if (b == R(0)) return mu0 * (-expm1_r(-a * dt));
    R k = a + b;
    R e = exp_r(-k * dt);
    R mu = k * mu0 * e / (k - b * mu0 * (R(1) - e));
    return mu0 - mu;
}

__device__ __forceinline__ int map_index(int j, int n, int bc)
{
    if (bc == 0) {
        if (j < 0) j += n;
        if (j >= n) j -= n;
    }
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

// plane of the velocity with v_y reversed (orbits axis, diagonal, axis, diagonal:
// (c,0) (0,c) (-c,0) (0,-c) and (+,+) (-,+) (-,-) (+,-)); lambda maps to itself
__host__ __device__ __forceinline__ int mirror_plane(int p)
{
    return p == 16 ? 16 : (((p >> 2) & 1) ? ((p & ~3) | (3 - (p & 3))) : ((p & 1) ? (p ^ 2) : p));
}

// Value of plane p at (x, y) of the ghost-extended grid: inside the grid the stored
// value; outside it the side's condition: periodic wrap, zero gradient (and walls,
// corrected afterwards) copy the edge cell, Dirichlet gives the side's equilibrium,
// specular mirrors the cell across the face with v_y reversed. A Dirichlet y side
// wins in a corner (corner ghosts are never read by the cross-shaped stencils).
template <typename R>
__device__ __forceinline__ R ghost_value(const ModelConst<R>& K, const R* __restrict__ in, int p,
                                         int x, int y)
{
    int sp = p;
    if (y < 0 || y >= K.ny) {
        const int s = y < 0 ? 2 : 3, code = K.sbc[s];
        if (code == 3) return K.sfeq[s][p];
        if (code == 4) {
            y = y < 0 ? -y - 1 : 2 * K.ny - 1 - y;
            y = y < 0 ? 0 : (y >= K.ny ? K.ny - 1 : y);
            sp = mirror_plane(p);
        } else {
            y = map_index(y, K.ny, code == 0 ? 0 : 1);
        }
    }
    if (x < 0 || x >= K.nx) {
        const int s = x < 0 ? 0 : 1, code = K.sbc[s];
        if (code == 3) return K.sfeq[s][p];
        x = map_index(x, K.nx, code == 0 ? 0 : 1);
    }
    return in[sp * K.plane + (int64_t)y * K.pitch + x];
}

__device__ __forceinline__ float lane_recip(float x) { return 1.0f / x; }
__device__ __forceinline__ double lane_recip(double x) { return 1.0 / x; }

// Non-equilibrium extrapolation at a wall (Sec. IV.D): the ghost cell next to a wall
// is the adjacent fluid cell f plus d = M^-1 [f_hat^eq(rho, u_w, T_w) - f_hat^eq(rho,
// u, T)], with rho, u, T those of f (plain sums in the lane type) and u_w, T_w the
// wall's (side 0 below row 0, side 1 above row ny-1).
template <typename R, typename L>
__device__ __forceinline__ void wall_correction(const ModelConst<R>& K, const L* f, int side, L* d)
{
    L m[16], qw[16], qs[16], dm[16];
    forward_moments(K, f, m);
    const L rho = m[0];
    const L ir = lane_recip(rho);
    const L ux = m[1] * ir, uy = m[2] * ir;
    const L T = (m[3] * ir - ux * ux - uy * uy) * K.inv_DI;
    feq_moments(L(K.DI), rho, L(K.wux[side]), L(K.wuy[side]), L(K.wT[side]), qw);
    feq_moments(L(K.DI), rho, ux, uy, T, qs);
#pragma unroll
    for (int k = 0; k < 16; k++) dm[k] = qw[k] - qs[k];
    inverse_moments(K, dm, d);
}



} // namespace lbk
