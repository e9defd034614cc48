// d2v24.cu -- the paper's own 24-velocity model (D2V24, Sec. II Eqs. (25)-(27)):
// kernels and the C ABI of include/lbkm24.h.
//
// The step is one fused kernel per time step, one thread per cell: the 24 f_i of
// the cell and of its NND stencil (radius 2 in x and y) are read through the
// read-only data cache; rho, u, T of the block's cells and a one-cell rim are formed
// once, in FP64 (an FP32 state sums its conserved moments as exact double-floats on
// the FP32 pipes first), and kept in shared memory; the equilibrium moments, the 20
// non-conserved moments, the relaxation, the back-transform, the chemical term of
// Eq. (24) and the NND update run in the storage type R (FP64 or FP32); the TNE
// partials of the state being read are reduced per block when due (sums in FP64,
// extremes exactly in R), and an 82-block kernel turns them into one history record.
//
// M and M^-1 act in block form: butterflies inside each orbit of four velocities
// (axis: f1+f3, f2+f4, f1-f3, f2-f4; diagonal: the sum and the three sign patterns)
// split the 24 components by parity in (v_x, v_y), and the moments of each parity
// sector depend on that sector's components only. The sectors are 9 (even, even:
// m1 m4 m5 m7 m14 m16 m17 m19 m20), 6 (odd, even: m2 m8 m10 m12 m21 m23), 6 (even,
// odd: m3 m9 m11 m13 m22 m24) and 3 (odd, odd: m6 m15 m18), so one transform costs
// 162 multiply-adds instead of 576. The blocks and their inverses are built on the
// host from M itself (checking that everything outside the blocks vanishes) and
// reach the kernel as kernel-parameter (constant-bank) operands.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "cell.cuh"
#include "kernels.cuh"
#include "lbkm24.h"
#include "pair.cuh"

namespace v24 {

using lbk::DevCounters;
using lbk::f2d_exact;
using lbk::map_index;
using lbk::nnd_neg;
using lbk::nnd_pos;
using lbk::reaction_increment;

constexpr int NV = 24;
constexpr int NP = NV + 1;       // planes: f_1..f_24, lambda
constexpr int TK = NV - 4;       // non-conserved moments Delta_5..Delta_24
constexpr int NQ = 4 * TK + 2;   // TNE quantities: sum, |sum|, min, max of each, d, d^2
constexpr int BT = 128;          // threads per block: 128 x 1 or 32 x 1 (1-D grids), 32 x 4
constexpr int MAC_CELLS = 390;   // macros staged per block: (128 + 2) x 3 >= (32 + 2) x 6
constexpr int GRAPH_CHUNK = 32;  // even: a replay leaves the ping-pong index unchanged

// signs of v_x, v_y of velocity i = 8 g + 4 o + j (speed group g, o = 0 axis orbit with
// (1,0) (0,1) (-1,0) (0,-1), o = 1 diagonal orbit with (1,1) (-1,1) (-1,-1) (1,-1)); the
// speeds are positive, so the upwind side of every plane is fixed at compile time
__host__ __device__ constexpr int vsign_x(int i)
{
    return ((i >> 2) & 1) == 0 ? ((i & 3) == 0 ? 1 : ((i & 3) == 2 ? -1 : 0))
                               : (((i & 3) == 0 || (i & 3) == 3) ? 1 : -1);
}
__host__ __device__ constexpr int vsign_y(int i)
{
    return ((i >> 2) & 1) == 0 ? ((i & 3) == 1 ? 1 : ((i & 3) == 3 ? -1 : 0)) : ((i & 3) < 2 ? 1 : -1);
}

// parity sectors: sizes, offsets of their blocks, and the moment (0-based) at each
// sector-ordered position p = 0..23 (ee 0..8, oe 9..14, eo 15..20, oo 21..23)
constexpr int NSEC = 4;
constexpr int NB = 162; // 81 + 36 + 36 + 9 block entries
__host__ __device__ constexpr int sec_n(int s) { return s == 0 ? 9 : (s == 3 ? 3 : 6); }
__host__ __device__ constexpr int sec_p(int s) { return s == 0 ? 0 : (s == 1 ? 9 : (s == 2 ? 15 : 21)); }
__host__ __device__ constexpr int sec_b(int s) { return s == 0 ? 0 : (s == 1 ? 81 : (s == 2 ? 117 : 153)); }
__host__ __device__ constexpr int mom_of(int p)
{
    constexpr int t[NV] = {0, 3, 4, 6, 13, 15, 16, 18, 19, 1, 7, 9, 11, 20, 22,
                           2, 8, 10, 12, 21, 23, 5, 14, 17};
    return t[p];
}

struct Record {
    double sum[NV], abs_sum[NV], min[NV], max[NV];
    double d_sum, d2_sum;
    int64_t step;
};
static_assert(sizeof(Record) == sizeof(lbkm24_tne_global), "record layout");

// Model constants, passed by value (constant bank). M is row-major [k][i]
// (moment k of velocity i), Minv row-major [i][k].
template <typename R>
struct Model {
    R Bf[NB];  // forward blocks, row-major [moment][component] per sector
    R Bi[NB];  // their inverses, row-major [component][moment]
    R vx[NV], vy[NV], eta2[NV], S[NV];
    R vxs[NV], vys[NV];              // v_x / dx and v_y / dy in R
    R dt_r, inv_dx_r, inv_dy_r, hdx_r, hdy_r, I_r, DI_r, A8c_r, A9c_r; // constants in R
    double vxd[NV], vyd[NV], wd[NV]; // FP64 copies for the conserved sums
    double cd[6], wod[6];            // speed and v^2 + eta^2 of each orbit (FP64)
    float cdh[6], cdl[6], wdh[6], wdl[6]; // the same split into hi + lo FP32 pairs
    double Minvd[NV * NV];           // FP64 M^-1 for the equilibrium start
    double I, DI, inv_DI, Q, omega1, omega2, T_ig, A8c, A9c;
    double dt, inv_dx, inv_dy;
    int nx, ny, pitch, bc_x, bc_y, pad_;
    int64_t plane;
    // per-side conditions (bc_x or bc_y = LBKM_BC_SIDES) of the sides x = 0, x = nx,
    // y = 0, y = ny: 1 zero gradient, 3 Dirichlet (ghost cells hold sfeq: the
    // equilibrium f of the side's state and its lambda), 4 specular (y sides: the mirror
    // cell across the face with v_y reversed); 0 for a periodic direction
    int sbc[4];
    R sfeq[4][NP];
    // walls (code 2, y sides) by non-equilibrium extrapolation: the ghost rows take the
    // edge row's f plus wall[side][i][x] = [M^-1 (f_hat^eq(rho, u_w, T_w) -
    // f_hat^eq(rho, u, T))]_i, rho, u, T of the edge cell, refreshed before every step
    const R* wall;
    double wux[2], wuy[2], wT[2];
};

struct Args {
    const void* in;
    void* out;
    double* partials;  // [NQ][grid blocks]
    DevCounters* ctr;
    Record* hist;
    int hist_cap;
    int tne_every;
    double area;       // dx * dy
};

__device__ __forceinline__ double tcomb(int kind, double a, double b)
{
    return kind == 0 ? a + b : (kind == 1 ? fmin(a, b) : fmax(a, b));
}
// quantity q: [0, TK) sum, [TK, 2TK) |.| sum, [2TK, 3TK) min, [3TK, 4TK) max, 4TK d, 4TK+1 d^2
__host__ __device__ __forceinline__ int tkind(int q)
{
    return (q < 2 * TK || q >= 4 * TK) ? 0 : (q < 3 * TK ? 1 : 2);
}

// FP64 -> R: exact (double) or rounded to nearest on the integer pipe (float)
template <typename R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_r<float>(double x) { return lbk::d2f_rn(x); }

__device__ __forceinline__ double to_f64(double x) { return x; }
// exact, on the integer pipe (the FP64 unit runs at 1/58 of the FP32 rate on GB300)
__device__ __forceinline__ double to_f64(float x) { return f2d_exact(x); }

// plane of the velocity with v_y reversed (axis orbits (c,0) (0,c) (-c,0) (0,-c);
// diagonal orbits (+,+) (-,+) (-,-) (+,-)); lambda maps to itself
__host__ __device__ __forceinline__ int mirror24(int i)
{
    if (i >= NV) return i;
    const int o = i / 4, j = i % 4;
    const int jm = (o & 1) ? 3 - j : (j == 1 ? 3 : (j == 3 ? 1 : j));
    return 4 * o + jm;
}

// Value of plane i (0..23 f, 24 lambda) at cell (x, y), which may lie up to two cells
// outside the grid: periodic or zero-gradient directions map the index; with per-side
// conditions a Dirichlet side (a y side first, as corners are never read by the
// cross-shaped stencil) gives its equilibrium value, a specular y side the mirror
// cell's value of the velocity with v_y reversed, an outflow side the edge cell's.
template <typename R>
__device__ __forceinline__ R fval(const Model<R>& K, const R* __restrict__ in, int i, int x, int y)
{
    const int cx = (x >= 0 && x < K.nx) ? -1 : (K.bc_x == 5 ? K.sbc[x < 0 ? 0 : 1] : K.bc_x);
    const int cy = (y >= 0 && y < K.ny) ? -1 : (K.bc_y == 5 ? K.sbc[y < 0 ? 2 : 3] : K.bc_y);
    if (cy == 3) return K.sfeq[y < 0 ? 2 : 3][i];
    if (cx == 3) return K.sfeq[x < 0 ? 0 : 1][i];
    const int sx = cx == -1 ? x : map_index(x, K.nx, cx == 0 ? 0 : 1);
    if (cy == 2) { // wall: the edge row plus its non-equilibrium correction (lambda copied)
        const int side = y < 0 ? 0 : 1, sy = side ? K.ny - 1 : 0;
        const R edge = __ldg(in + (size_t)i * K.plane + (size_t)sy * K.pitch + sx);
        return i < NV ? edge + K.wall[((size_t)side * NV + i) * K.nx + sx] : edge;
    }
    int sy, ii = i;
    if (cy == 4) {
        sy = y < 0 ? -y - 1 : 2 * K.ny - 1 - y;
        ii = mirror24(i);
    } else {
        sy = cy == -1 ? y : map_index(y, K.ny, cy == 0 ? 0 : 1);
    }
    return __ldg(in + (size_t)ii * K.plane + (size_t)sy * K.pitch + sx);
}

// rho, u_x, u_y and, if asked, T (FP64) at cell (x, y) of state `in`, boundary conditions
// applied (Eqs. (5)-(7)). The sums go orbit by orbit: an orbit of speed c adds its sum s
// to rho, c times its x and y differences to rho u, and (c^2 or 2 c^2) + eta^2 times s to
// the energy moment m_4; 1/rho comes from an FP32 seed and two Newton steps.
template <typename R, bool GEN = false>
__device__ __forceinline__ void conserved_at(const Model<R>& K, const R* __restrict__ in, int x,
                                             int y, double& rho, double& ux, double& uy,
                                             double* T = nullptr)
{
    R gf[GEN ? NV : 1];
    if constexpr (GEN) {
#pragma unroll
        for (int i = 0; i < NV; i++) gf[i] = fval(K, in, i, x, y);
    }
    x = map_index(x, K.nx, K.bc_x == 0 ? 0 : 1);
    y = map_index(y, K.ny, K.bc_y == 0 ? 0 : 1);
    const R* p = in + (size_t)y * K.pitch + x;
    // plane i of this cell: through the side rules, or straight from the mapped cell
    auto ld = [&](int i) -> R {
        if constexpr (GEN) return gf[i];
        else return __ldg(p + (size_t)i * K.plane);
    };
    double r = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
    if constexpr (sizeof(R) == 4) {
        // FP32 state: the same sums as double-floats on the FP32 pipes (error-free
        // TwoSum butterflies, products with split constants, ~48 significant bits),
        // carried into FP64 once
        using lbk::df;
        df R0{0.f, 0.f}, R1{0.f, 0.f}, R2{0.f, 0.f}, R3{0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 6; o++) {
            const float a = ld(4 * o), b = ld(4 * o + 1), c = ld(4 * o + 2), d = ld(4 * o + 3);
            const df sac = lbk::two_sum(a, c), sbd = lbk::two_sum(b, d);
            const df dac = lbk::two_sum(a, -c), dbd = lbk::two_sum(b, -d);
            const df sum = lbk::df_add(sac, sbd);
            df gx = dac, gy = dbd;
            if (o & 1) {
                gx = lbk::df_sub(dac, dbd);
                gy = lbk::df_add(dac, dbd);
            }
            const df co{K.cdh[o], K.cdl[o]};
            R0 = lbk::df_add(R0, sum);
            R1 = lbk::df_add(R1, lbk::df_mul(co, gx));
            R2 = lbk::df_add(R2, lbk::df_mul(co, gy));
            if (T) R3 = lbk::df_add(R3, lbk::df_mul(df{K.wdh[o], K.wdl[o]}, sum));
        }
        r = f2d_exact(R0.hi) + f2d_exact(R0.lo);
        jx = f2d_exact(R1.hi) + f2d_exact(R1.lo);
        jy = f2d_exact(R2.hi) + f2d_exact(R2.lo);
        if (T) e = f2d_exact(R3.hi) + f2d_exact(R3.lo);
    } else {
#pragma unroll
    for (int o = 0; o < 6; o++) {
        const double a = to_f64(ld(4 * o)), b = to_f64(ld(4 * o + 1));
        const double c = to_f64(ld(4 * o + 2)), d = to_f64(ld(4 * o + 3));
        const double sac = a + c, sbd = b + d, dac = a - c, dbd = b - d;
        const double sum = sac + sbd;
        double gx, gy;
        if ((o & 1) == 0) { // axis: (1,0) (0,1) (-1,0) (0,-1)
            gx = dac;
            gy = dbd;
        } else {            // diagonal: (1,1) (-1,1) (-1,-1) (1,-1)
            gx = dac - dbd;
            gy = dac + dbd;
        }
        r += sum;
        jx = fma(K.cd[o], gx, jx);
        jy = fma(K.cd[o], gy, jy);
        if (T) e = fma(K.wod[o], sum, e);
    }
    }
    double q = f2d_exact(lbk::rcp_approx(lbk::d2f_rn(r)));
    q = fma(q, fma(-r, q, 1.0), q);
    q = fma(q, fma(-r, q, 1.0), q);
    rho = r;
    ux = jx * q;
    uy = jy * q;
    if (T) *T = (e * q - (ux * ux + uy * uy)) * K.inv_DI;
}

// orbit butterflies: f (velocity order) -> g (sector order)
template <typename R>
__host__ __device__ __forceinline__ void butterfly(const R* f, R* g)
{
#pragma unroll
    for (int o = 0; o < 6; o++) {
        const R a = f[4 * o], b = f[4 * o + 1], c = f[4 * o + 2], d = f[4 * o + 3];
        const int e0 = (o / 2) * 3;
        if ((o & 1) == 0) { // axis orbit: (1,0) (0,1) (-1,0) (0,-1)
            g[e0] = a + c;
            g[e0 + 1] = b + d;
            g[9 + o] = a - c;
            g[15 + o] = b - d;
        } else {            // diagonal orbit: (1,1) (-1,1) (-1,-1) (1,-1)
            g[e0 + 2] = (a + c) + (b + d);
            g[9 + o] = (a - c) - (b - d);
            g[15 + o] = (a - c) + (b - d);
            g[21 + o / 2] = (a + c) - (b + d);
        }
    }
}

// inverse butterflies: g (sector order) -> f (velocity order)
template <typename R>
__host__ __device__ __forceinline__ void unbutterfly(const R* g, R* f)
{
#pragma unroll
    for (int o = 0; o < 6; o++) {
        const int e0 = (o / 2) * 3;
        if ((o & 1) == 0) {
            const R sx = g[e0], sy = g[e0 + 1], ax = g[9 + o], ay = g[15 + o];
            f[4 * o] = R(0.5) * (sx + ax);
            f[4 * o + 1] = R(0.5) * (sy + ay);
            f[4 * o + 2] = R(0.5) * (sx - ax);
            f[4 * o + 3] = R(0.5) * (sy - ay);
        } else {
            const R e = g[e0 + 2], ax = g[9 + o], ay = g[15 + o], od = g[21 + o / 2];
            f[4 * o] = R(0.25) * ((e + od) + (ax + ay));
            f[4 * o + 1] = R(0.25) * ((e - od) - (ax - ay));
            f[4 * o + 2] = R(0.25) * ((e + od) - (ax + ay));
            f[4 * o + 3] = R(0.25) * ((e - od) + (ax - ay));
        }
    }
}

// y = blockdiag(B) x over the four sectors (x, y in sector order)
template <typename R>
__device__ __forceinline__ void block_apply(const R* B, const R* x, R* y)
{
#pragma unroll
    for (int sct = 0; sct < NSEC; sct++) {
        const int n = sec_n(sct), p0 = sec_p(sct), b0 = sec_b(sct);
#pragma unroll
        for (int r = 0; r < n; r++) {
            R acc = R(0);
#pragma unroll
            for (int j = 0; j < n; j++) acc = fma(B[b0 + r * n + j], x[p0 + j], acc);
            y[p0 + r] = acc;
        }
    }
}

// f_hat^eq_1..24 (list after Eq. (16); entries 14 and 16 with the factor T of Eq. (11)),
// in the arithmetic type F
template <typename F>
__host__ __device__ __forceinline__ void feq24(F I, F DI, F rho, F ux, F uy, F T, F* q)
{
    const F u2 = ux * ux + uy * uy;
    const F A = (DI + F(2)) * T + u2, B = (DI + F(4)) * T + u2;
    const F rx = rho * ux, ry = rho * uy, IT = I * T;
    const F C = u2 * u2 + F(4) * (DI + F(4)) * T * T + (DI + F(10)) * u2 * T; // D = 2
    q[0] = rho;
    q[1] = rx;
    q[2] = ry;
    q[3] = rho * (DI * T + u2);
    q[4] = rho * (T + ux * ux);
    q[5] = rx * uy;
    q[6] = rho * (T + uy * uy);
    q[7] = rx * A;
    q[8] = ry * A;
    q[9] = rx * (F(3) * T + ux * ux);
    q[10] = ry * (T + ux * ux);
    q[11] = rx * (T + uy * uy);
    q[12] = ry * (F(3) * T + uy * uy);
    q[13] = rho * A * T + rx * ux * B;
    q[14] = rx * uy * B;
    q[15] = rho * A * T + ry * uy * B;
    q[16] = rho * IT * (T + ux * ux);
    q[17] = rx * uy * IT;
    q[18] = rho * IT * (T + uy * uy);
    q[19] = rho * IT * (u2 + (F(2) + F(3) * I) * T);
    q[20] = rx * C;
    q[21] = ry * C;
    q[22] = rx * IT * (u2 + (F(4) + F(3) * I) * T);
    q[23] = ry * IT * (u2 + (F(4) + F(3) * I) * T);
}

// Block reduction of the TNE quantities of the block's cells into partials
// [q * nblocks + b], q in the record's order (sums of Delta_k, of |Delta_k|, minima,
// maxima, sum of d, sum of d^2). Each thread leaves its cell's Delta_5..24, d and d^2
// (formed in R) in shared memory; each quantity is then reduced in three parts of a
// third of the block's cells (one thread per part; the block's threads take the parts
// in turn), in a fixed order: the 42 sums exactly (FP64, or FP32 TwoSum pairs for an
// FP32 state), the 40 extremes in R (exact); one thread per quantity joins the three
// parts in FP64. Deterministic for any block size <= BT.
template <typename R>
__device__ __forceinline__ void block_tne(const R* Dk, bool active, double* partials, int nblocks,
                                          int b)
{
    constexpr int LD = BT + 1;            // padded rows: the readers walk along a row
    constexpr int NS = 2 * TK + 2;        // sums: Delta_k, |Delta_k|, d, d^2
    constexpr int NE = 2 * TK;            // extremes: min and max of Delta_k
    __shared__ R sD[TK + 2][LD];
    __shared__ unsigned char sact[BT];
    __shared__ double spart[NQ][3];
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    const int per = (nt + 2) / 3; // cells per part
    R d2 = R(0);
#pragma unroll
    for (int k = 0; k < TK; k++) {
        sD[k][t] = Dk[k];
        d2 = fma(Dk[k], Dk[k], d2);
    }
    sD[TK][t] = sqrt(d2);
    sD[TK + 1][t] = d2;
    sact[t] = active ? 1 : 0;
    __syncthreads();
    for (int w = t; w < 3 * NS; w += nt) {
        const int s = w / 3, part = w - 3 * s;
        const int q = s < 2 * TK ? s : 4 * TK + (s - 2 * TK);
        const int row = s < TK ? s : (s < 2 * TK ? s - TK : TK + (s - 2 * TK));
        const bool absv = s >= TK && s < 2 * TK;
        const int j1 = min((part + 1) * per, nt);
        if constexpr (sizeof(R) == 4) {
            // FP32 terms summed exactly: each addition's rounding error (TwoSum) goes to
            // a compensating term, the pair joined in FP64 once (the FP64 unit runs at
            // 1/58 of the FP32 rate on this part)
            float sum = 0.f, comp = 0.f;
            for (int j = part * per; j < j1; j++) {
                if (!sact[j]) continue;
                const float v = absv ? fabsf(sD[row][j]) : sD[row][j];
                const lbk::df t2 = lbk::two_sum(sum, v);
                sum = t2.hi;
                comp += t2.lo;
            }
            spart[q][part] = (double)sum + (double)comp;
        } else {
            double acc = 0.0;
            for (int j = part * per; j < j1; j++) {
                if (!sact[j]) continue;
                const double v = (double)sD[row][j];
                acc += absv ? fabs(v) : v;
            }
            spart[q][part] = acc;
        }
    }
    for (int w = t; w < 3 * NE; w += nt) {
        const int e = w / 3, part = w - 3 * e;
        const bool mn = e < TK;
        const int k = mn ? e : e - TK;
        const int j1 = min((part + 1) * per, nt);
        bool any = false;
        R m = R(0);
        for (int j = part * per; j < j1; j++) {
            if (!sact[j]) continue;
            const R v = sD[k][j];
            m = !any ? v : (mn ? fmin(m, v) : fmax(m, v));
            any = true;
        }
        spart[2 * TK + e][part] = any ? (double)m : (mn ? DBL_MAX : -DBL_MAX);
    }
    __syncthreads();
    for (int q = t; q < NQ; q += nt) {
        const int kind = tkind(q);
        partials[(size_t)q * nblocks + b] =
            tcomb(kind, tcomb(kind, spart[q][0], spart[q][1]), spart[q][2]);
    }
}

// SRT: the single-relaxation-time fast path (all R_5..R_24 equal, no TNE due): with one
// rate the moment-space relaxation is -R (f - M^-1 f_hat^eq) in velocity space (the SRT
// form of Sec. V) and A_hat vanishes, so the forward transform of f is skipped and only
// f^eq = M^-1 f_hat^eq is formed (it also feeds the chemical term of Eq. (24)).
template <typename R, bool SRT, bool GEN>
__global__ void __launch_bounds__(BT, sizeof(R) == 4 ? 3 : 1) step_kernel(const Model<R> K, const Args a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = x < K.nx && y < K.ny;
    const int64_t step = a.ctr->step;
    const bool do_tne = !SRT && a.tne_every > 0 && (step % a.tne_every) == 0;
    const R* __restrict__ in = static_cast<const R*>(a.in);
    R* __restrict__ out = static_cast<R*>(a.out);
    R Dk[TK];
#pragma unroll
    for (int k = 0; k < TK; k++) Dk[k] = R(0);
    bool bad = false;

    // 1. conserved sums and macros in FP64 (Eqs. (5)-(7)) of the block's cells and a
    //    one-cell rim (the central differences of u need them), each computed once
    __shared__ double s_rho[MAC_CELLS], s_ux[MAC_CELLS], s_uy[MAC_CELLS], s_T[MAC_CELLS];
    {
        const int bw = blockDim.x + 2, bh = K.ny > 1 ? blockDim.y + 2 : 1;
        const int x0 = blockIdx.x * blockDim.x - 1, y0 = blockIdx.y * blockDim.y - (K.ny > 1);
        for (int c = threadIdx.x + threadIdx.y * blockDim.x; c < bw * bh;
             c += blockDim.x * blockDim.y) {
            const int hx = c % bw, hy = c / bw;
            conserved_at<R, GEN>(K, in, x0 + hx, y0 + hy, s_rho[c], s_ux[c], s_uy[c], &s_T[c]);
        }
        __syncthreads();
    }
    if (active) {
        const size_t g = (size_t)y * K.pitch + x;
        R f[NV];
#pragma unroll
        for (int i = 0; i < NV; i++) f[i] = __ldg(in + (size_t)i * K.plane + g);
        const R lam0 = __ldg(in + (size_t)NV * K.plane + g);

        const int bw = blockDim.x + 2, two = K.ny > 1;
        const int c0 = (threadIdx.y + two) * bw + threadIdx.x + 1;
        const double rho = s_rho[c0], ux = s_ux[c0], uy = s_uy[c0];
        const double T = s_T[c0];
        bad = !(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T);

        const double pT = rho * T;

        // 2. rho, u, T were recovered in FP64; the bulk from here on runs in R, including
        //    the velocity gradients (second-order central differences)
        const R rr = to_r<R>(rho), uxr = to_r<R>(ux), uyr = to_r<R>(uy), Tr = to_r<R>(T);
        const R Ir = K.I_r;
        const R gxx = (to_r<R>(s_ux[c0 + 1]) - to_r<R>(s_ux[c0 - 1])) * K.hdx_r;
        const R gyx = (to_r<R>(s_uy[c0 + 1]) - to_r<R>(s_uy[c0 - 1])) * K.hdx_r;
        R gxy = R(0), gyy = R(0);
        if (two) {
            gxy = (to_r<R>(s_ux[c0 + bw]) - to_r<R>(s_ux[c0 - bw])) * K.hdy_r;
            gyy = (to_r<R>(s_uy[c0 + bw]) - to_r<R>(s_uy[c0 - bw])) * K.hdy_r;
        }

        // 3. moments (block form), equilibrium moments, non-equilibrium parts
        R q[NV];
        feq24<R>(Ir, K.DI_r, rr, uxr, uyr, Tr, q);
        if (!SRT) {
            R gv[NV], h[NV];
            butterfly(f, gv);
            block_apply(K.Bf, gv, h);
#pragma unroll
            for (int p = 0; p < NV; p++)
                if (mom_of(p) >= 4) Dk[mom_of(p) - 4] = h[p] - q[mom_of(p)];
        }

        // 4. relaxation with A_hat_8, A_hat_9 (Eqs. (3)-(4), sign as in Eq. (29))
        R Om_hat[TK];
#pragma unroll
        for (int k = 0; k < TK; k++) Om_hat[k] = -K.S[k + 4] * Dk[k];
        if (!SRT) {
            const R th = (gxx + gyy) / K.DI_r, pTr = rr * Tr, shear = gyx + gxy;
            Om_hat[3] += pTr * K.A8c_r * (R(4) * uxr * (gxx - th) + R(2) * uyr * shear);
            Om_hat[4] += pTr * K.A9c_r * (R(4) * uyr * (gyy - th) + R(2) * uxr * shear);
        }

        // 5. reaction over dt with p and T frozen at t_n (Eq. (28), m = n = 1)
        double dlam = 0.0;
        if (T > K.T_ig)
            dlam = reaction_increment<double>((double)lam0, K.omega1 * pT, K.omega2 * pT, K.dt);
        const double lrate = dlam / K.dt;

        // 6. back-transform (block form), chemical term of Eq. (24) on f^eq = M^-1 f_hat^eq,
        //    NND advection, forward Euler
        const bool react = lrate != 0.0;
        R Om[NV], fe[NV];
        {
            R w[NV], gv[NV];
            if (!SRT) {
#pragma unroll
                for (int p = 0; p < NV; p++) w[p] = mom_of(p) >= 4 ? Om_hat[mom_of(p) - 4] : R(0);
                block_apply(K.Bi, w, gv);
                unbutterfly(gv, Om);
            }
            if (SRT || react) {
#pragma unroll
                for (int p = 0; p < NV; p++) w[p] = q[mom_of(p)];
                block_apply(K.Bi, w, gv);
                unbutterfly(gv, fe);
            }
            if (SRT) {
#pragma unroll
                for (int i = 0; i < NV; i++) Om[i] = -K.S[4] * (f[i] - fe[i]);
            }
        }
        const R chem = react ? to_r<R>(K.Q * lrate / (K.I * K.DI * T * T)) : R(0);
        const R base = R(-3) * Ir * Tr; // -(1 + D) I T
        const int xm2 = map_index(x - 2, K.nx, K.bc_x == 0 ? 0 : 1);
        const int xm1 = map_index(x - 1, K.nx, K.bc_x == 0 ? 0 : 1);
        const int xp1 = map_index(x + 1, K.nx, K.bc_x == 0 ? 0 : 1);
        const int xp2 = map_index(x + 2, K.nx, K.bc_x == 0 ? 0 : 1);
        const int by = K.bc_y == 0 ? 0 : 1;
        const size_t row = (size_t)y * K.pitch;
        const size_t ym2 = (size_t)map_index(y - 2, K.ny, by) * K.pitch;
        const size_t ym1 = (size_t)map_index(y - 1, K.ny, by) * K.pitch;
        const size_t yp1 = (size_t)map_index(y + 1, K.ny, by) * K.pitch;
        const size_t yp2 = (size_t)map_index(y + 2, K.ny, by) * K.pitch;
        // stencil value of plane i at x + d (LX) or y + d (LY): the side rules for the
        // per-side variant, the mapped offsets otherwise
        auto LX = [&](int i, int d) -> R {
            if constexpr (GEN) return fval(K, in, i, x + d, y);
            const int xo = d == -2 ? xm2 : (d == -1 ? xm1 : (d == 1 ? xp1 : xp2));
            return __ldg(in + (size_t)i * K.plane + row + xo);
        };
        auto LY = [&](int i, int d) -> R {
            if constexpr (GEN) return fval(K, in, i, x, y + d);
            const size_t yo = d == -2 ? ym2 : (d == -1 ? ym1 : (d == 1 ? yp1 : yp2));
            return __ldg(in + (size_t)i * K.plane + yo + x);
        };
#pragma unroll
        for (int i = 0; i < NV; i++) {
            R om = Om[i];
            if (react) {
                const R cx = K.vx[i] - uxr, cy = K.vy[i] - uyr;
                om += fe[i] * chem * (base + Ir * (cx * cx + cy * cy) + K.eta2[i]);
            }
            const R* pl = in + (size_t)i * K.plane;
            R adv = R(0);
            if (vsign_x(i) > 0)
                adv = K.vxs[i] * nnd_pos(LX(i, -2), LX(i, -1), f[i], LX(i, 1));
            else if (vsign_x(i) < 0)
                adv = K.vxs[i] * nnd_neg(LX(i, -1), f[i], LX(i, 1), LX(i, 2));
            if (K.ny > 1) {
                if (vsign_y(i) > 0)
                    adv += K.vys[i] * nnd_pos(LY(i, -2), LY(i, -1), f[i], LY(i, 1));
                else if (vsign_y(i) < 0)
                    adv += K.vys[i] * nnd_neg(LY(i, -1), f[i], LY(i, 1), LY(i, 2));
            }
            out[(size_t)i * K.plane + g] = f[i] + K.dt_r * (om - adv);
        }

        // 7. lambda: u . grad(lambda) with NND interface values, then the update
        R la = R(0);
        if (uxr > R(0))
            la = uxr * K.inv_dx_r * nnd_pos(LX(NV, -2), LX(NV, -1), lam0, LX(NV, 1));
        else if (uxr < R(0))
            la = uxr * K.inv_dx_r * nnd_neg(LX(NV, -1), lam0, LX(NV, 1), LX(NV, 2));
        if (K.ny > 1) {
            if (uyr > R(0))
                la += uyr * K.inv_dy_r * nnd_pos(LY(NV, -2), LY(NV, -1), lam0, LY(NV, 1));
            else if (uyr < R(0))
                la += uyr * K.inv_dy_r * nnd_neg(LY(NV, -1), lam0, LY(NV, 1), LY(NV, 2));
        }
        R ln = lam0 - K.dt_r * la + to_r<R>(dlam);
        ln = ln < R(0) ? R(0) : (ln > R(1) ? R(1) : ln);
        out[(size_t)NV * K.plane + g] = ln;
    }

    // TNE partials of the state read (all threads take part), status, step counter
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    const int b = blockIdx.x + blockIdx.y * gridDim.x, nb = gridDim.x * gridDim.y;
    if (do_tne) block_tne(Dk, active, a.partials, nb, b);
    if (__syncthreads_or(bad) && t == 0) atomicOr(&a.ctr->status, 1);
    __shared__ unsigned int s_last;
    if (t == 0) s_last = (atomicAdd(&a.ctr->arrivals, 1u) == (unsigned)nb - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last && t == 0) {
        if (do_tne) {
            a.ctr->hist_count += 1;
            a.ctr->tne_step = step;
        }
        a.ctr->tne_pending = do_tne ? 1 : 0;
        a.ctr->step = step + 1;
        a.ctr->arrivals = 0u;
    }
}

// TNE of a state on demand: Delta fields (optional) and block partials.
template <typename R>
__global__ void __launch_bounds__(BT) tne_kernel(const Model<R> K, const R* __restrict__ in,
                                                 double* delta, double* partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = x < K.nx && y < K.ny;
    R Dk[TK];
#pragma unroll
    for (int k = 0; k < TK; k++) Dk[k] = R(0);
    if (active) {
        const size_t g = (size_t)y * K.pitch + x;
        double rho, ux, uy, T;
        conserved_at(K, in, x, y, rho, ux, uy, &T);
        R q[NV];
        feq24<R>(K.I_r, K.DI_r, to_r<R>(rho), to_r<R>(ux), to_r<R>(uy), to_r<R>(T), q);
        R f[NV], gv[NV], h[NV];
#pragma unroll
        for (int i = 0; i < NV; i++) f[i] = __ldg(in + (size_t)i * K.plane + g);
        butterfly(f, gv);
        block_apply(K.Bf, gv, h);
#pragma unroll
        for (int p = 0; p < NV; p++)
            if (mom_of(p) >= 4) Dk[mom_of(p) - 4] = h[p] - q[mom_of(p)];
        if (delta) {
            const size_t n = (size_t)K.nx * K.ny, c = (size_t)y * K.nx + x;
#pragma unroll
            for (int k = 0; k < NV; k++) delta[k * n + c] = k < 4 ? 0.0 : (double)Dk[k - 4];
        }
    }
    block_tne(Dk, active, partials, gridDim.x * gridDim.y, blockIdx.x + blockIdx.y * gridDim.x);
}

// Record of a grid's partials: block q reduces quantity q in a fixed order.
// rec == nullptr: the step's record, into history slot (hist_count - 1) % cap,
// only when the step left partials (ctr->tne_pending).
__global__ void __launch_bounds__(256)
    finish_kernel(const double* __restrict__ partials, int nblocks, Record* hist, int hist_cap,
                  const DevCounters* ctr, Record* rec_out, double area)
{
    if (!rec_out && !ctr->tne_pending) return;
    __shared__ double wsum[8];
    const int q = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int kind = tkind(q);
    double acc = kind == 0 ? 0.0 : (kind == 1 ? DBL_MAX : -DBL_MAX);
    const double* pq = partials + (size_t)q * nblocks;
    for (int b = t; b < nblocks; b += 256) acc = tcomb(kind, acc, __ldcg(pq + b));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = tcomb(kind, acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) wsum[w] = acc;
    __syncthreads();
    if (t != 0) return;
    for (int k = 1; k < 8; k++) acc = tcomb(kind, acc, wsum[k]);
    Record* rec = rec_out ? rec_out : hist + (ctr->hist_count - 1) % hist_cap;
    if (q < TK) rec->sum[q + 4] = acc * area;
    else if (q < 2 * TK) rec->abs_sum[q - TK + 4] = acc * area;
    else if (q < 3 * TK) rec->min[q - 2 * TK + 4] = acc;
    else if (q < 4 * TK) rec->max[q - 3 * TK + 4] = acc;
    else if (q == 4 * TK) rec->d_sum = acc * area;
    else rec->d2_sum = acc * area;
    if (q == 0) {
        for (int k = 0; k < 4; k++) rec->sum[k] = rec->abs_sum[k] = rec->min[k] = rec->max[k] = 0.0;
        rec->step = rec_out ? ctr->step : ctr->tne_step;
    }
}

// The wall corrections of the edge rows (non-equilibrium extrapolation, Sec. IV.D):
// thread (side, x) forms rho, u, T of the edge cell in FP64 and
// M^-1 [f_hat^eq(rho, u_w, T_w) - f_hat^eq(rho, u, T)] in FP64, stored in R.
template <typename R>
__global__ void wall_kernel(const Model<R> K, const R* __restrict__ in, R* wall)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * K.nx) return;
    const int side = t / K.nx, x = t % K.nx;
    if (K.sbc[2 + side] != 2) return;
    double rho, ux, uy, T;
    conserved_at<R, false>(K, in, x, side ? K.ny - 1 : 0, rho, ux, uy, &T);
    double qw[NV], qf[NV];
    feq24<double>(K.I, K.DI, rho, K.wux[side], K.wuy[side], K.wT[side], qw);
    feq24<double>(K.I, K.DI, rho, ux, uy, T, qf);
#pragma unroll 4
    for (int i = 0; i < NV; i++) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < NV; k++) acc = fma(K.Minvd[i * NV + k], qw[k] - qf[k], acc);
        wall[((size_t)side * NV + i) * K.nx + x] = (R)acc;
    }
}

template <typename R>
__global__ void init_kernel(const Model<R> K, const double* rho, const double* ux,
                            const double* uy, const double* T, const double* lam, R* state)
{
    const int64_t n = (int64_t)K.nx * K.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % K.nx), y = (int)(c / K.nx);
        double q[NV];
        feq24<double>(K.I, K.DI, rho[c], ux[c], uy[c], T[c], q);
        const size_t g = (size_t)y * K.pitch + x;
#pragma unroll
        for (int i = 0; i < NV; i++) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < NV; k++) s = fma(K.Minvd[i * NV + k], q[k], s);
            state[(size_t)i * K.plane + g] = (R)s;
        }
        state[(size_t)NV * K.plane + g] = lam ? (R)lam[c] : R(0);
    }
}

template <typename R>
__global__ void macros_kernel(const Model<R> K, const R* __restrict__ in, double* rho,
                              double* ux, double* uy, double* T, double* p, double* lam)
{
    const int64_t n = (int64_t)K.nx * K.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % K.nx), y = (int)(c / K.nx);
        double r, u, v, t;
        conserved_at(K, in, x, y, r, u, v, &t);
        if (rho) rho[c] = r;
        if (ux) ux[c] = u;
        if (uy) uy[c] = v;
        if (T) T[c] = t;
        if (p) p[c] = r * t;
        if (lam) lam[c] = (double)in[(size_t)NV * K.plane + (size_t)y * K.pitch + x];
    }
}

// ---------------------------------------------------------------- host side

// velocities of the paper's D2V24 (Eqs. (25)-(27))
void velocity_table(const double v[3], const double eta[3], double* vx, double* vy, double* e)
{
    static const int AX[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    static const int DG[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int g = 0; g < 3; g++)
        for (int o = 0; o < 2; o++)
            for (int j = 0; j < 4; j++) {
                const int i = 8 * g + 4 * o + j;
                vx[i] = v[g] * (o == 0 ? AX[j][0] : DG[j][0]);
                vy[i] = v[g] * (o == 0 ? AX[j][1] : DG[j][1]);
                e[i] = eta[g];
            }
}

// rows m_1..m_24 (list after Eq. (16)) at the discrete velocities
void moment_rows(const double* vx, const double* vy, const double* e, double* M)
{
    for (int i = 0; i < NV; i++) {
        const double a = vx[i], b = vy[i], e2 = e[i] * e[i], v2 = a * a + b * b, w = v2 + e2;
        const double col[NV] = {1.0,       a,         b,         w,         a * a,
                                a * b,     b * b,     w * a,     w * b,     a * a * a,
                                a * a * b, a * b * b, b * b * b, w * a * a, w * a * b,
                                w * b * b, e2 * a * a, e2 * a * b, e2 * b * b, w * e2,
                                w * v2 * a, w * v2 * b, w * e2 * a, w * e2 * b};
        for (int k = 0; k < NV; k++) M[k * NV + i] = col[k];
    }
}

// The inverse of an n x n matrix (n <= 24) by LU factorisation with partial pivoting
// in long double, one step of iterative refinement per column. Returns max |A Ainv - 1|,
// or -1 if singular.
double invert(const double* M, double* Minv, int n = NV)
{
    long double lu[NV][NV];
    int perm[NV];
    long double amax = 0;
    for (int r = 0; r < n; r++) {
        perm[r] = r;
        for (int c = 0; c < n; c++) {
            lu[r][c] = M[r * n + c];
            amax = fmaxl(amax, fabsl(lu[r][c]));
        }
    }
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int r = k + 1; r < n; r++)
            if (fabsl(lu[r][k]) > fabsl(lu[p][k])) p = r;
        if (fabsl(lu[p][k]) < 1e-13L * amax) return -1.0;
        if (p != k) {
            for (int c = 0; c < n; c++) {
                long double t = lu[k][c];
                lu[k][c] = lu[p][c];
                lu[p][c] = t;
            }
            int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
        }
        for (int r = k + 1; r < n; r++) {
            lu[r][k] /= lu[k][k];
            for (int c = k + 1; c < n; c++) lu[r][c] -= lu[r][k] * lu[k][c];
        }
    }
    auto solve = [&](const long double* rhs, long double* x) {
        long double z[NV];
        for (int r = 0; r < n; r++) {
            long double s = rhs[perm[r]];
            for (int c = 0; c < r; c++) s -= lu[r][c] * z[c];
            z[r] = s;
        }
        for (int r = n - 1; r >= 0; r--) {
            long double s = z[r];
            for (int c = r + 1; c < n; c++) s -= lu[r][c] * x[c];
            x[r] = s / lu[r][r];
        }
    };
    for (int col = 0; col < n; col++) {
        long double e[NV], x[NV], res[NV], dx[NV];
        for (int r = 0; r < n; r++) e[r] = r == col ? 1.0L : 0.0L;
        solve(e, x);
        for (int r = 0; r < n; r++) {
            long double s = e[r];
            for (int c = 0; c < n; c++) s -= (long double)M[r * n + c] * x[c];
            res[r] = s;
        }
        solve(res, dx);
        for (int r = 0; r < n; r++) Minv[r * n + col] = (double)(x[r] + dx[r]);
    }
    double worst = 0.0;
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            long double s = 0;
            for (int k = 0; k < n; k++) s += (long double)M[r * n + k] * Minv[k * n + c];
            worst = fmax(worst, fabs((double)(s - (r == c ? 1.0L : 0.0L))));
        }
    return worst;
}

// The sector blocks of M (column j of a sector = M applied to the inverse butterfly of
// that sector's j-th unit component, restricted to the sector's moments) and their
// inverses. Returns the largest |entry| M produces outside the blocks relative to the
// largest inside, or -1 if a block is singular.
double build_blocks(const double* M, double* Bf, double* Bi)
{
    double leak = 0.0, big = 0.0;
    for (int sct = 0; sct < NSEC; sct++) {
        const int n = sec_n(sct), p0 = sec_p(sct);
        double blk[NV * NV], inv[NV * NV];
        for (int j = 0; j < n; j++) {
            double gv[NV] = {0}, f[NV], col[NV];
            gv[p0 + j] = 1.0;
            unbutterfly(gv, f);
            for (int k = 0; k < NV; k++) {
                col[k] = 0.0;
                for (int i = 0; i < NV; i++) col[k] += M[k * NV + i] * f[i];
            }
            for (int p = 0; p < NV; p++) {
                const bool inside = p >= p0 && p < p0 + n;
                if (inside) {
                    blk[(p - p0) * n + j] = col[mom_of(p)];
                    big = fmax(big, fabs(col[mom_of(p)]));
                } else {
                    leak = fmax(leak, fabs(col[mom_of(p)]));
                }
            }
        }
        const double res = invert(blk, inv, n);
        if (res < 0.0 || res > 1e-9) return -1.0;
        for (int k = 0; k < n * n; k++) {
            Bf[sec_b(sct) + k] = blk[k];
            Bi[sec_b(sct) + k] = inv[k];
        }
    }
    return leak / big;
}

template <typename R>
void fill_model(const lbkm24_params& p, const double* Bf, const double* Bi, const double* Minv,
                const double* vx, const double* vy, const double* e, int pitch,
                const int* sbc, const double (*sfeq)[NP], Model<R>* K)
{
    memset(K, 0, sizeof(*K));
    for (int sd = 0; sd < 4; sd++) {
        K->sbc[sd] = sbc[sd];
        for (int i = 0; i < NP; i++) K->sfeq[sd][i] = (R)sfeq[sd][i];
    }
    for (int k = 0; k < NB; k++) {
        K->Bf[k] = (R)Bf[k];
        K->Bi[k] = (R)Bi[k];
    }
    for (int k = 0; k < NV * NV; k++) K->Minvd[k] = Minv[k];
    for (int i = 0; i < NV; i++) {
        K->vx[i] = (R)vx[i];
        K->vy[i] = (R)vy[i];
        K->eta2[i] = (R)(e[i] * e[i]);
        K->S[i] = (R)p.S[i];
        K->vxd[i] = vx[i];
        K->vyd[i] = vy[i];
        K->wd[i] = vx[i] * vx[i] + vy[i] * vy[i] + e[i] * e[i];
    }
    for (int o = 0; o < 6; o++) {
        const double c = p.v[o / 2], et = p.eta[o / 2];
        K->cd[o] = c;
        K->wod[o] = c * c * ((o & 1) ? 2.0 : 1.0) + et * et;
        K->cdh[o] = (float)c;
        K->cdl[o] = (float)(c - (double)K->cdh[o]);
        K->wdh[o] = (float)K->wod[o];
        K->wdl[o] = (float)(K->wod[o] - (double)K->wdh[o]);
    }
    K->I = 2.0 / (p.gamma - 1.0) - 2.0;
    K->DI = 2.0 + K->I;
    K->inv_DI = 1.0 / K->DI;
    K->Q = p.Q;
    K->omega1 = p.omega1;
    K->omega2 = p.omega2;
    K->T_ig = p.T_ig;
    K->A8c = (p.S[4] - p.S[7]) / p.S[4];
    K->A9c = (p.S[6] - p.S[8]) / p.S[6];
    K->dt = p.dt;
    K->inv_dx = 1.0 / p.dx;
    K->inv_dy = 1.0 / p.dy;
    for (int i = 0; i < NV; i++) {
        K->vxs[i] = (R)(vx[i] / p.dx);
        K->vys[i] = (R)(vy[i] / p.dy);
    }
    K->dt_r = (R)p.dt;
    K->inv_dx_r = (R)(1.0 / p.dx);
    K->inv_dy_r = (R)(1.0 / p.dy);
    K->hdx_r = (R)(0.5 / p.dx);
    K->hdy_r = (R)(0.5 / p.dy);
    K->I_r = (R)K->I;
    K->DI_r = (R)K->DI;
    K->A8c_r = (R)K->A8c;
    K->A9c_r = (R)K->A9c;
    K->nx = p.nx;
    K->ny = p.ny;
    K->pitch = pitch;
    K->bc_x = p.bc_x;
    K->bc_y = p.bc_y;
    K->plane = (int64_t)pitch * p.ny;
}

thread_local std::string g_create_error;

} // namespace v24

using namespace v24;

struct lbkm24 {
    lbkm24_params p;
    Model<double> Kd;
    Model<float> Kf;
    int pitch;
    size_t elem, plane_elems;
    cudaStream_t stream, capture_stream;
    void* buf[2];
    int cur;
    double* partials;
    int nblocks;
    dim3 grid, block;
    DevCounters* ctr;
    Record* hist;
    Record* tne_out;
    bool initialized;
    bool srt;  // the single-relaxation-time fast path runs the steps
    bool has_wall;
    void* wallbuf;  // [2][24][nx] wall corrections in the state's precision
    int64_t host_steps;
    cudaGraphExec_t graph[2];
    std::string err;
};

namespace {

lbkm_status fail(lbkm24_t h, lbkm_status st, const char* fmt, ...)
{
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof(b), fmt, ap);
    va_end(ap);
    (h ? h->err : g_create_error) = b;
    return st;
}

#define TRY24(h, call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((h), e_ == cudaErrorMemoryAllocation ? LBKM_ENOMEM : LBKM_ECUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

cudaError_t launch_one_step(const lbkm24* h, int from, cudaStream_t st)
{
    Args a;
    a.in = h->buf[from];
    a.out = h->buf[1 - from];
    a.partials = h->partials;
    a.ctr = h->ctr;
    a.hist = h->hist;
    a.hist_cap = h->p.tne_capacity;
    a.tne_every = h->p.tne_every;
    a.area = h->p.dx * h->p.dy;
    const bool gen = h->p.bc_x == LBKM_BC_SIDES || h->p.bc_y == LBKM_BC_SIDES;
    if (h->has_wall) {
        const int g = (2 * h->p.nx + 127) / 128;
        if (h->p.precision == LBKM_F64)
            wall_kernel<double><<<g, 128, 0, st>>>(h->Kd, (const double*)a.in, (double*)h->wallbuf);
        else
            wall_kernel<float><<<g, 128, 0, st>>>(h->Kf, (const float*)a.in, (float*)h->wallbuf);
        const cudaError_t we = cudaGetLastError();
        if (we != cudaSuccess) return we;
    }
#define V24_LAUNCH(R_, KK)                                                                   \
    do {                                                                                     \
        if (h->srt && gen) step_kernel<R_, true, true><<<h->grid, h->block, 0, st>>>(KK, a); \
        else if (h->srt) step_kernel<R_, true, false><<<h->grid, h->block, 0, st>>>(KK, a);  \
        else if (gen) step_kernel<R_, false, true><<<h->grid, h->block, 0, st>>>(KK, a);     \
        else step_kernel<R_, false, false><<<h->grid, h->block, 0, st>>>(KK, a);             \
    } while (0)
    if (h->p.precision == LBKM_F64)
        V24_LAUNCH(double, h->Kd);
    else
        V24_LAUNCH(float, h->Kf);
#undef V24_LAUNCH
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && h->p.tne_every > 0) {
        finish_kernel<<<NQ, 256, 0, st>>>(h->partials, h->nblocks, h->hist, h->p.tne_capacity,
                                          h->ctr, nullptr, a.area);
        e = cudaGetLastError();
    }
    return e;
}

// streaming multiprocessors of the current device (152 on GB300, the value taken if the
// query fails)
int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return 152;
    }
    return sms;
}

int elementwise_blocks(int64_t n)
{
    const int64_t b = (n + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

lbkm_status check(lbkm24_t h)
{
    TRY24(h, cudaStreamSynchronize(h->stream));
    int st = 0;
    TRY24(h, cudaMemcpy(&st, &h->ctr->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 1)
        return fail(h, LBKM_EUNSTABLE,
                    "a cell reached a non-finite or non-positive density or temperature");
    return LBKM_OK;
}

void to_global(const Record& r, lbkm24_tne_global* g) { memcpy(g, &r, sizeof(r)); }

} // namespace

extern "C" {

void lbkm24_default_params(lbkm24_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->precision = LBKM_F64;
    p->gamma = 1.4;
    p->v[0] = 2.7;
    p->v[1] = 2.2;
    p->v[2] = 1.2;
    p->eta[0] = 5.0;
    p->eta[1] = 3.0;
    p->eta[2] = 1.1;
    for (int k = 0; k < NV; k++) p->S[k] = (k >= 4 && k <= 6) ? 1e4 : 1e5;
    p->Q = 1.0;
    p->T_ig = 1.1;
    p->dx = p->dy = 2e-4;
    p->dt = 5e-6;
    p->bc_x = LBKM_BC_ZERO_GRADIENT;
    p->bc_y = LBKM_BC_PERIODIC;
    p->tne_capacity = 1;
}

const char* lbkm24_last_error(lbkm24_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

lbkm_status lbkm24_create(const lbkm24_params* pin, void* cuda_stream, lbkm24_t* out)
{
    if (!out) return fail(nullptr, LBKM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!pin) return fail(nullptr, LBKM_EINVAL, "params is NULL");
    const lbkm24_params& p = *pin;
    if (p.nx < 1 || p.ny < 1 || (int64_t)p.nx * p.ny > (int64_t)1 << 30)
        return fail(nullptr, LBKM_EINVAL, "nx, ny must be >= 1 (at most 2^30 cells)");
    if (p.precision != LBKM_F64 && p.precision != LBKM_F32)
        return fail(nullptr, LBKM_EINVAL, "precision must be LBKM_F64 or LBKM_F32");
    if (!(p.gamma > 1.0) || !(2.0 / (p.gamma - 1.0) - 2.0 > 0.0))
        return fail(nullptr, LBKM_EINVAL, "gamma must give I = 2/(gamma-1) - 2 > 0");
    for (int g = 0; g < 3; g++) {
        if (!(p.v[g] > 0.0) || !isfinite(p.v[g]))
            return fail(nullptr, LBKM_EINVAL, "v[%d] must be finite and > 0", g);
        if (!(p.eta[g] >= 0.0) || !isfinite(p.eta[g]))
            return fail(nullptr, LBKM_EINVAL, "eta[%d] must be finite and >= 0", g);
    }
    double smax = 0.0;
    for (int k = 4; k < NV; k++) {
        if (!(p.S[k] > 0.0) || !isfinite(p.S[k]))
            return fail(nullptr, LBKM_EINVAL, "S[%d] must be finite and > 0", k);
        smax = fmax(smax, p.S[k]);
    }
    if (!(p.dx > 0) || !(p.dy > 0) || !(p.dt > 0))
        return fail(nullptr, LBKM_EINVAL, "dx, dy, dt must be > 0");
    if (!(p.dt * smax < 2.0))
        return fail(nullptr, LBKM_EINVAL, "dt * max S = %g must be < 2", p.dt * smax);
    const double vmax = fmax(p.v[0], fmax(p.v[1], p.v[2])); // per-axis component of the diagonals
    const double cfl = vmax * p.dt * (1.0 / p.dx + (p.ny > 1 ? 1.0 / p.dy : 0.0));
    if (!(cfl <= 1.0))
        return fail(nullptr, LBKM_EINVAL, "CFL number %g of the fastest velocity exceeds 1", cfl);
    if (!(p.omega1 >= 0) || !(p.omega2 >= 0) || !isfinite(p.Q))
        return fail(nullptr, LBKM_EINVAL, "omega1, omega2 must be >= 0 and Q finite");
    if (!(p.T_ig >= 0) || !isfinite(p.T_ig))
        return fail(nullptr, LBKM_EINVAL, "T_ig must be finite and >= 0");
    for (int d = 0; d < 2; d++) {
        const int bc = d == 0 ? p.bc_x : p.bc_y;
        if (bc != LBKM_BC_PERIODIC && bc != LBKM_BC_ZERO_GRADIENT && bc != LBKM_BC_SIDES)
            return fail(nullptr, LBKM_EINVAL, "%s must be periodic, zero gradient or sides",
                        d == 0 ? "bc_x" : "bc_y");
    }
    for (int sd = 0; sd < 4; sd++) {
        if ((sd < 2 ? p.bc_x : p.bc_y) != LBKM_BC_SIDES) continue;
        const int code = p.side_bc[sd];
        const bool ok = code == LBKM_BC_ZERO_GRADIENT || code == LBKM_BC_DIRICHLET ||
                        ((code == LBKM_BC_SPECULAR || code == LBKM_BC_WALL) && sd >= 2);
        if (!ok)
            return fail(nullptr, LBKM_EINVAL,
                        "side_bc[%d]: zero gradient, Dirichlet, or specular / wall (y sides only)",
                        sd);
        if ((code == LBKM_BC_SPECULAR || code == LBKM_BC_WALL) && p.ny < 2)
            return fail(nullptr, LBKM_EINVAL, "a specular or wall side needs ny >= 2");
        if (code == LBKM_BC_WALL &&
            (!(p.side_T[sd] > 0) || !isfinite(p.side_T[sd]) || !isfinite(p.side_ux[sd]) ||
             !isfinite(p.side_uy[sd])))
            return fail(nullptr, LBKM_EINVAL, "side %d: a wall needs T > 0 and a finite velocity",
                        sd);
        if (code == LBKM_BC_DIRICHLET &&
            (!(p.side_rho[sd] > 0) || !(p.side_T[sd] > 0) || !isfinite(p.side_rho[sd]) ||
             !isfinite(p.side_T[sd]) || !isfinite(p.side_ux[sd]) || !isfinite(p.side_uy[sd]) ||
             !(p.side_lam[sd] >= 0 && p.side_lam[sd] <= 1)))
            return fail(nullptr, LBKM_EINVAL,
                        "side %d: Dirichlet state needs rho > 0, T > 0, finite u, lambda in [0, 1]",
                        sd);
    }
    if (p.tne_every < 0 || (p.tne_every > 0 && p.tne_capacity < 1))
        return fail(nullptr, LBKM_EINVAL, "tne_every >= 0 and tne_capacity >= 1");
    if (p.collision != 0 && p.collision != 1)
        return fail(nullptr, LBKM_EINVAL, "collision must be 0 (fast path allowed) or 1");

    double vx[NV], vy[NV], e[NV], M[NV * NV], Minv[NV * NV], Bf[NB], Bi[NB];
    velocity_table(p.v, p.eta, vx, vy, e);
    moment_rows(vx, vy, e, M);
    const double res = invert(M, Minv);
    const double leak = res < 0.0 ? -1.0 : build_blocks(M, Bf, Bi);
    if (res < 0.0 || res > 1e-9 || leak < 0.0)
        return fail(nullptr, LBKM_ESINGULAR, "the D2V24 velocity set gives a singular M");
    if (leak > 1e-12)
        return fail(nullptr, LBKM_ESINGULAR, "M is not block-diagonal under the butterflies");

    lbkm24* h = new lbkm24();
    h->p = p;
    if (h->p.tne_capacity < 1) h->p.tne_capacity = 1;
    h->stream = (cudaStream_t)cuda_stream;
    h->elem = p.precision == LBKM_F64 ? 8 : 4;
    h->pitch = (p.nx + 31) / 32 * 32;
    h->plane_elems = (size_t)h->pitch * p.ny;
    bool equal = true;
    for (int k = 5; k < NV; k++) equal = equal && p.S[k] == p.S[4];
    h->srt = equal && p.tne_every == 0 && p.collision == 0;
    // Dirichlet sides: ghost f = M^-1 f_hat^eq(side state), ghost lambda = the side's
    int sbc[4] = {0, 0, 0, 0};
    double sfeq[4][NP];
    memset(sfeq, 0, sizeof(sfeq));
    const double Ih = 2.0 / (p.gamma - 1.0) - 2.0;
    for (int sd = 0; sd < 4; sd++) {
        if ((sd < 2 ? p.bc_x : p.bc_y) != LBKM_BC_SIDES) continue;
        sbc[sd] = p.side_bc[sd];
        if (sbc[sd] != LBKM_BC_DIRICHLET) continue;
        double q[NV];
        feq24<double>(Ih, 2.0 + Ih, p.side_rho[sd], p.side_ux[sd], p.side_uy[sd], p.side_T[sd], q);
        for (int i = 0; i < NV; i++) {
            double acc = 0.0;
            for (int k = 0; k < NV; k++) acc += Minv[i * NV + k] * q[k];
            sfeq[sd][i] = acc;
        }
        sfeq[sd][NV] = p.side_lam[sd];
    }
    fill_model(p, Bf, Bi, Minv, vx, vy, e, h->pitch, sbc, sfeq, &h->Kd);
    fill_model(p, Bf, Bi, Minv, vx, vy, e, h->pitch, sbc, sfeq, &h->Kf);
    h->has_wall = p.bc_y == LBKM_BC_SIDES && (sbc[2] == LBKM_BC_WALL || sbc[3] == LBKM_BC_WALL);
    for (int w = 0; w < 2; w++) {
        h->Kd.wux[w] = h->Kf.wux[w] = p.side_ux[2 + w];
        h->Kd.wuy[w] = h->Kf.wuy[w] = p.side_uy[2 + w];
        h->Kd.wT[w] = h->Kf.wT[w] = p.side_T[2 + w];
    }
    // 1-D grids too short to give every SM a block of 128 cells run blocks of one warp:
    // the step is latency-bound there, and more SMs each take fewer cells
    const bool narrow = p.ny == 1 && (p.nx + BT - 1) / BT < 2 * sm_count();
    h->block = p.ny > 1 ? dim3(32, BT / 32) : dim3(narrow ? 32 : BT, 1);
    h->grid = dim3((p.nx + h->block.x - 1) / h->block.x, (p.ny + h->block.y - 1) / h->block.y);
    h->nblocks = (int)(h->grid.x * h->grid.y);
    auto bail = [&](cudaError_t ce, const char* what) {
        lbkm24_destroy(h);
        return fail(nullptr, ce == cudaErrorMemoryAllocation ? LBKM_ENOMEM : LBKM_ECUDA, "%s: %s",
                    what, cudaGetErrorString(ce));
    };
    cudaError_t ce;
    const size_t sb = (size_t)NP * h->plane_elems * h->elem;
    for (int k = 0; k < 2; k++)
        if ((ce = cudaMalloc(&h->buf[k], sb)) != cudaSuccess) return bail(ce, "state");
    if ((ce = cudaMalloc((void**)&h->partials, sizeof(double) * NQ * h->nblocks)) != cudaSuccess)
        return bail(ce, "partials");
    if (h->has_wall) {
        const size_t wb = sizeof(double) * 2 * NV * (size_t)p.nx;
        if ((ce = cudaMalloc(&h->wallbuf, wb)) != cudaSuccess) return bail(ce, "walls");
        if ((ce = cudaMemset(h->wallbuf, 0, wb)) != cudaSuccess) return bail(ce, "walls");
        h->Kd.wall = static_cast<const double*>(h->wallbuf);
        h->Kf.wall = static_cast<const float*>(h->wallbuf);
    }
    if ((ce = cudaMalloc((void**)&h->ctr, sizeof(DevCounters))) != cudaSuccess)
        return bail(ce, "counters");
    if ((ce = cudaMalloc((void**)&h->hist, sizeof(Record) * h->p.tne_capacity)) != cudaSuccess)
        return bail(ce, "history");
    if ((ce = cudaMalloc((void**)&h->tne_out, sizeof(Record))) != cudaSuccess)
        return bail(ce, "record");
    if ((ce = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(ce, "capture stream");
    if ((ce = cudaMemset(h->buf[0], 0, sb)) != cudaSuccess ||
        (ce = cudaMemset(h->buf[1], 0, sb)) != cudaSuccess ||
        (ce = cudaMemset(h->ctr, 0, sizeof(DevCounters))) != cudaSuccess)
        return bail(ce, "clear");
    *out = h;
    return LBKM_OK;
}

void lbkm24_destroy(lbkm24_t h)
{
    if (!h) return;
    if (h->stream || h->buf[0]) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 2; i++) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        if (h->buf[i]) cudaFree(h->buf[i]);
    }
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->partials) cudaFree(h->partials);
    if (h->ctr) cudaFree(h->ctr);
    if (h->hist) cudaFree(h->hist);
    if (h->tne_out) cudaFree(h->tne_out);
    if (h->wallbuf) cudaFree(h->wallbuf);
    delete h;
}

lbkm_status lbkm24_init_fields(lbkm24_t h, const double* rho, const double* ux, const double* uy,
                               const double* T, const double* lambda, int on_device)
{
    if (!h) return LBKM_EINVAL;
    if (!rho || !ux || !uy || !T) return fail(h, LBKM_EINVAL, "rho, ux, uy and T are required");
    const size_t n = (size_t)h->p.nx * h->p.ny, nb = n * sizeof(double);
    const double* src[5] = {rho, ux, uy, T, lambda};
    const double* dev[5] = {rho, ux, uy, T, lambda};
    double* tmp = nullptr;
    if (!on_device) {
        TRY24(h, cudaMallocAsync((void**)&tmp, nb * 5, h->stream));
        for (int k = 0; k < 5; k++) {
            if (!src[k]) {
                dev[k] = nullptr;
                continue;
            }
            TRY24(h, cudaMemcpyAsync(tmp + k * n, src[k], nb, cudaMemcpyHostToDevice, h->stream));
            dev[k] = tmp + k * n;
        }
    }
    const int g = elementwise_blocks((int64_t)n);
    if (h->p.precision == LBKM_F64)
        init_kernel<double><<<g, 256, 0, h->stream>>>(h->Kd, dev[0], dev[1], dev[2], dev[3],
                                                      dev[4], (double*)h->buf[0]);
    else
        init_kernel<float><<<g, 256, 0, h->stream>>>(h->Kf, dev[0], dev[1], dev[2], dev[3],
                                                     dev[4], (float*)h->buf[0]);
    TRY24(h, cudaGetLastError());
    h->cur = 0;
    TRY24(h, cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), h->stream));
    if (tmp) TRY24(h, cudaFreeAsync(tmp, h->stream));
    TRY24(h, cudaStreamSynchronize(h->stream));
    h->initialized = true;
    h->host_steps = 0;
    return LBKM_OK;
}

lbkm_status lbkm24_step(lbkm24_t h, int64_t n)
{
    if (!h) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm24_step before lbkm24_init_fields");
    if (n < 0) return fail(h, LBKM_EINVAL, "n must be >= 0");
    while (n >= GRAPH_CHUNK) {
        cudaGraphExec_t& ex = h->graph[h->cur];
        if (!ex) {
            cudaGraph_t gr;
            TRY24(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t le = cudaSuccess;
            for (int s = 0; s < GRAPH_CHUNK && le == cudaSuccess; s++)
                le = launch_one_step(h, (h->cur + s) & 1, h->capture_stream);
            cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &gr);
            if (le != cudaSuccess || ce != cudaSuccess) {
                if (ce == cudaSuccess) cudaGraphDestroy(gr);
                return fail(h, LBKM_ECUDA, "graph capture: %s",
                            cudaGetErrorString(le != cudaSuccess ? le : ce));
            }
            cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
            cudaGraphDestroy(gr);
            if (ie != cudaSuccess)
                return fail(h, LBKM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
        }
        TRY24(h, cudaGraphLaunch(ex, h->stream));
        n -= GRAPH_CHUNK;
        h->host_steps += GRAPH_CHUNK;
    }
    for (; n > 0; n--) {
        TRY24(h, launch_one_step(h, h->cur, h->stream));
        h->cur = 1 - h->cur;
        h->host_steps++;
    }
    return LBKM_OK;
}

lbkm_status lbkm24_sync(lbkm24_t h)
{
    if (!h) return LBKM_EINVAL;
    return check(h);
}

int64_t lbkm24_steps_taken(lbkm24_t h) { return h ? h->host_steps : -1; }

lbkm_status lbkm24_macros(lbkm24_t h, double* rho, double* ux, double* uy, double* T, double* p,
                          double* lambda, int on_device)
{
    if (!h) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm24_macros before lbkm24_init_fields");
    const size_t n = (size_t)h->p.nx * h->p.ny, nb = n * sizeof(double);
    double* outs[6] = {rho, ux, uy, T, p, lambda};
    double* dev[6] = {rho, ux, uy, T, p, lambda};
    double* tmp = nullptr;
    if (!on_device) {
        TRY24(h, cudaMallocAsync((void**)&tmp, nb * 6, h->stream));
        for (int k = 0; k < 6; k++) dev[k] = outs[k] ? tmp + k * n : nullptr;
    }
    const int g = elementwise_blocks((int64_t)n);
    if (h->p.precision == LBKM_F64)
        macros_kernel<double><<<g, 256, 0, h->stream>>>(h->Kd, (const double*)h->buf[h->cur],
                                                        dev[0], dev[1], dev[2], dev[3], dev[4],
                                                        dev[5]);
    else
        macros_kernel<float><<<g, 256, 0, h->stream>>>(h->Kf, (const float*)h->buf[h->cur], dev[0],
                                                       dev[1], dev[2], dev[3], dev[4], dev[5]);
    TRY24(h, cudaGetLastError());
    if (!on_device) {
        for (int k = 0; k < 6; k++)
            if (outs[k])
                TRY24(h, cudaMemcpyAsync(outs[k], dev[k], nb, cudaMemcpyDeviceToHost, h->stream));
        TRY24(h, cudaFreeAsync(tmp, h->stream));
    }
    return check(h);
}

lbkm_status lbkm24_tne(lbkm24_t h, double* delta, lbkm24_tne_global* g, int on_device)
{
    if (!h) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm24_tne before lbkm24_init_fields");
    const size_t n = (size_t)h->p.nx * h->p.ny, nb = (size_t)NV * n * sizeof(double);
    double* dd = delta;
    double* tmp = nullptr;
    if (delta && !on_device) {
        TRY24(h, cudaMallocAsync((void**)&tmp, nb, h->stream));
        dd = tmp;
    }
    if (h->p.precision == LBKM_F64)
        tne_kernel<double><<<h->grid, h->block, 0, h->stream>>>(
            h->Kd, (const double*)h->buf[h->cur], dd, h->partials);
    else
        tne_kernel<float><<<h->grid, h->block, 0, h->stream>>>(
            h->Kf, (const float*)h->buf[h->cur], dd, h->partials);
    TRY24(h, cudaGetLastError());
    finish_kernel<<<NQ, 256, 0, h->stream>>>(h->partials, h->nblocks, nullptr, 1, h->ctr,
                                             h->tne_out, h->p.dx * h->p.dy);
    TRY24(h, cudaGetLastError());
    if (tmp) {
        TRY24(h, cudaMemcpyAsync(delta, tmp, nb, cudaMemcpyDeviceToHost, h->stream));
        TRY24(h, cudaFreeAsync(tmp, h->stream));
    }
    Record r;
    TRY24(h, cudaMemcpyAsync(&r, h->tne_out, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    lbkm_status st = check(h);
    if (st != LBKM_OK) return st;
    if (g) to_global(r, g);
    return LBKM_OK;
}

lbkm_status lbkm24_tne_history(lbkm24_t h, lbkm24_tne_global* out, int32_t max_records,
                               int32_t* n_out)
{
    if (!h || !n_out || (max_records > 0 && !out)) return LBKM_EINVAL;
    *n_out = 0;
    lbkm_status st = check(h);
    if (st != LBKM_OK) return st;
    DevCounters c;
    TRY24(h, cudaMemcpy(&c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost));
    const int cap = h->p.tne_capacity;
    const int64_t have = c.hist_count < cap ? c.hist_count : cap;
    const int64_t take = have < max_records ? have : max_records;
    for (int64_t k = 0; k < take; k++) {
        Record r;
        TRY24(h, cudaMemcpy(&r, h->hist + (c.hist_count - have + k) % cap, sizeof(r),
                            cudaMemcpyDeviceToHost));
        to_global(r, out + k);
    }
    *n_out = (int32_t)take;
    return LBKM_OK;
}

size_t lbkm24_state_bytes(lbkm24_t h)
{
    return h ? (size_t)NP * h->p.nx * h->p.ny * h->elem + sizeof(int64_t) : 0;
}

lbkm_status lbkm24_get_state(lbkm24_t h, void* dst, int on_device)
{
    if (!h || !dst) return LBKM_EINVAL;
    if (!h->initialized) return fail(h, LBKM_ESTATE, "lbkm24_get_state before init_fields");
    const size_t row = (size_t)h->p.nx * h->elem, plane = row * h->p.ny;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int pl = 0; pl < NP; pl++)
        TRY24(h, cudaMemcpy2DAsync((char*)dst + pl * plane, row,
                                   (const char*)h->buf[h->cur] + pl * h->plane_elems * h->elem,
                                   h->pitch * h->elem, row, h->p.ny, k, h->stream));
    const int64_t s = h->host_steps;
    TRY24(h, cudaMemcpyAsync((char*)dst + NP * plane, &s, sizeof(s),
                             on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                             h->stream));
    return check(h);
}

lbkm_status lbkm24_set_state(lbkm24_t h, const void* src, int on_device)
{
    if (!h || !src) return LBKM_EINVAL;
    const size_t row = (size_t)h->p.nx * h->elem, plane = row * h->p.ny;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    h->cur = 0;
    for (int pl = 0; pl < NP; pl++)
        TRY24(h, cudaMemcpy2DAsync((char*)h->buf[0] + pl * h->plane_elems * h->elem,
                                   h->pitch * h->elem, (const char*)src + pl * plane, row, row,
                                   h->p.ny, k, h->stream));
    int64_t s = 0;
    TRY24(h, cudaMemcpyAsync(&s, (const char*)src + NP * plane, sizeof(s),
                             on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                             h->stream));
    TRY24(h, cudaStreamSynchronize(h->stream));
    DevCounters c;
    memset(&c, 0, sizeof(c));
    c.step = s;
    TRY24(h, cudaMemcpy(h->ctr, &c, sizeof(c), cudaMemcpyHostToDevice));
    h->host_steps = s;
    h->initialized = true;
    return LBKM_OK;
}

} // extern "C"
