// adjoint.cu -- discrete adjoint of the FP64 1-D step (reverse mode, hand-written).
//
// For one step (f, lambda)_n -> (f, lambda)_{n+1} of the fused kernel and adjoints
// (fb, lb)_{n+1} = dJ/d(state_{n+1}), these kernels produce (fb, lb)_n and add the
// step's contributions to dJ/dS_5..16, dJ/dQ, dJ/domega1, dJ/domega2. The forward
// values are recomputed from the stored FP64 state n (for an FP32 forward run, a state of
// the FP64 segment recomputed from the run's checkpoint, widened by adj_widen). Conventions at non-smooth points: the
// ignition switch T > T_ig is a hard switch (no derivative), minmod follows the
// branch the values select (a on a tie), the clamp of lambda passes the
// derivative when the unclamped value lies in [0, 1] (inclusive), the upwind
// choice for u.grad(lambda) by the sign of u has no derivative.
//
// Pass A (one thread per cell j): everything local to cell j -- back-transform
// (M^-T), relaxation (S, Delta), A_hat_8/9 (Eqs. (3)-(4)), reaction (Eq. (28)),
// chemical term (Eqs. (19)-(23)), f_hat^eq and its T-derivative, the lambda clamp
// and the local part of u.grad(lambda) -- giving adjoints of rho, u, T of cell j,
// of the velocity gradients gx, gy (which belong to the neighbours), of the
// non-conserved moments, of lambda, and the parameter partials.
// Pass A also forms, for each plane of its cell jp, the NND stencil's coefficients times
// the plane's upwind weight (-dt v f_b / dx for f_i, -dt u_x lambda_b / dx for lambda),
// one set per cell, branches decided by the forward values.
// Pass B (one thread per cell j): gathers what depends on neighbours -- the
// central differences of u, the transposed NND stencils of every f_i and of
// lambda (the coefficients that pass A left at the neighbours) -- then the macro
// chain rho, u, T <- conserved moments and M^T.
#include <float.h>
#include <math.h>

#include "adjoint.cuh"
#include "cell.cuh"
#include "kernels.cuh"

namespace lbk {

namespace {

__device__ __forceinline__ int bmap(int j, int n, int bc) { return map_index(j, n, bc); }

// the cell at distance d from j whose stencil may read j: its periodic image, or -1 past
// a zero-gradient end (nx >= 5 keeps the periodic candidates of d = -2..2 distinct)
__device__ __forceinline__ int neighbour(int j, int d, int n, int bc)
{
    const int jp = j + d;
    if (bc == 0) return jp < 0 ? jp + n : (jp >= n ? jp - n : jp);
    return jp < 0 || jp >= n ? -1 : jp;
}

// minmod branch of mm(a, b): alpha = derivative w.r.t. a, beta w.r.t. b
__device__ __forceinline__ void mm_branch(double a, double b, double& al, double& be)
{
    const bool same = a * b > 0.0;
    const bool first = fabs(a) <= fabs(b);
    al = (same && first) ? 1.0 : 0.0;
    be = (same && !first) ? 1.0 : 0.0;
}

// d(expr)/d(q at offsets -2..+2) of the NND flux difference of cell j for v > 0
// (uses offsets -2..+1) or v < 0 (offsets -1..+2); expr as in nnd_pos / nnd_neg.
__device__ __forceinline__ void nnd_coef(double vsign, const double* q, double* c)
{
    c[0] = c[1] = c[2] = c[3] = c[4] = 0.0;
    if (vsign > 0.0) {
        const double d0 = q[1] - q[0], d1 = q[2] - q[1], d2 = q[3] - q[2];
        double a01, b01, a12, b12;
        mm_branch(d0, d1, a01, b01);
        mm_branch(d1, d2, a12, b12);
        const double P = 1.0 + 0.5 * a12 - 0.5 * b01;
        c[0] = 0.5 * a01;
        c[1] = -P - 0.5 * a01;
        c[2] = P - 0.5 * b12;
        c[3] = 0.5 * b12;
    } else if (vsign < 0.0) {
        const double d1 = q[2] - q[1], d2 = q[3] - q[2], d3 = q[4] - q[3];
        double a12, b12, a23, b23;
        mm_branch(d1, d2, a12, b12);
        mm_branch(d2, d3, a23, b23);
        const double P = 1.0 - 0.5 * a23 + 0.5 * b12;
        c[1] = -0.5 * a12;
        c[2] = -P + 0.5 * a12;
        c[3] = P + 0.5 * b23;
        c[4] = -0.5 * b23;
    }
}

constexpr int ADJ_THREADS = 128;

// The increment of lambda over dt (Eq. (28), m = n = 1: the closed form of
// d lambda/dt = (1 - lambda)(a + b lambda), evaluated as the step evaluates it) and its
// partial derivatives with respect to lambda, a = omega1 p and b = omega2 p. With
// mu0 = 1 - lambda, k = a + b, e = exp(-k dt): mu = k mu0 e / (k - b mu0 (1 - e)) and
// dl = mu0 - mu; for b = 0, mu = mu0 e, whose derivative in b is the limit b -> 0.
__device__ __forceinline__ void reaction_partials(double lam, double a, double b, double dt,
                                                  double& dl, double& d_lam, double& d_a,
                                                  double& d_b)
{
    const double mu0 = 1.0 - lam;
    if (b == 0.0) {
        const double g = -expm1(-a * dt), e = 1.0 - g;
        const double ga = a > 0.0 ? g / a : dt; // (1 - e) / a
        dl = mu0 * g;
        d_lam = -g;
        d_a = mu0 * dt * e;
        d_b = mu0 * e * dt - mu0 * mu0 * e * ga;
        return;
    }
    const double k = a + b, e = exp(-k * dt), g = 1.0 - e;
    const double Dn = k - b * mu0 * g;
    const double mu = k * mu0 * e / Dn;
    const double mu_k = (mu0 * e * (1.0 - k * dt) - mu * (1.0 - b * mu0 * dt * e)) / Dn;
    const double mu_m0 = (k * e + mu * b * g) / Dn;
    dl = mu0 - mu;
    d_lam = mu_m0 - 1.0;
    d_a = -mu_k;
    d_b = -(mu_k + mu * mu0 * g / Dn);
}

// block sum of v in fixed order, added by thread 0 to acc[blockIdx.x]
__device__ void block_add(double v, double* acc, double* sred)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < ADJ_THREADS / 32; k++) s += sred[k];
        acc[blockIdx.x] += s;
    }
}

__global__ void __launch_bounds__(ADJ_THREADS)
    adj_pass_a(const ModelConst<double> K, const AdjArgs a)
{
    __shared__ double sred[ADJ_THREADS / 32];
    const int nx = K.nx;
    const double DI = K.DI, dt = K.dt;
    double pS[ADJ_NPAR];
    for (int q = 0; q < ADJ_NPAR; q++) pS[q] = 0.0;
    double jt = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx; j += gridDim.x * blockDim.x) {
        double f[16], m[16], q[16], dq[16];
        for (int i = 0; i < 16; i++) f[i] = a.f[i * K.plane + j];
        const double lam = a.f[16 * K.plane + j];
        const double rho = a.mac[j], ux = a.mac[nx + j], uy = a.mac[2 * nx + j],
                     T = a.mac[3 * nx + j];
        forward_moments(K, f, m);
        feq_moments(DI, rho, ux, uy, T, q);
        dfeq_dT(DI, rho, ux, uy, T, dq);
        double Dk[16];
        for (int k = 4; k < 16; k++) Dk[k] = m[k] - q[k];
        const int jl = bmap(j - 1, nx, K.bc_x), jr = bmap(j + 1, nx, K.bc_x);
        const double gx = (a.mac[nx + jr] - a.mac[nx + jl]) * K.half_inv_dx;
        const double gy = (a.mac[2 * nx + jr] - a.mac[2 * nx + jl]) * K.half_inv_dx;
        const double A8c = K.A8c, A9c = K.A9c;
        const double X8 = 4.0 * ux * gx * (1.0 - 1.0 / DI) + 2.0 * uy * gy;
        const double X9 = -4.0 * uy * gx / DI + 2.0 * ux * gy;
        // reaction over dt, decided by T > T_ig (Eq. (28))
        const bool ig = T > K.T_igd;
        const double pr = rho * T;
        double dl = 0.0, dl_lam = 0.0, dl_a = 0.0, dl_b = 0.0;
        if (ig) reaction_partials(lam, K.omega1 * pr, K.omega2 * pr, dt, dl, dl_lam, dl_a, dl_b);
        const double cr = dl * K.chem;
        // lambda update and its clamp
        double lq[5];
        for (int o = -2; o <= 2; o++) lq[o + 2] = a.f[16 * K.plane + bmap(j + o, nx, K.bc_x)];
        const double Lp = nnd_pos(lq[0], lq[1], lq[2], lq[3]);
        const double Ln = nnd_neg(lq[1], lq[2], lq[3], lq[4]);
        const double lsel = ux > 0.0 ? Lp : (ux < 0.0 ? Ln : 0.0);
        const double raw = lam - dt * (ux * lsel * K.inv_dx) + dl;
        const double lbc = (raw >= 0.0 && raw <= 1.0) ? a.lb1[j] : 0.0;
        // the weighted NND coefficients of this cell's stencils, for pass B to gather
        {
            double c[5];
            nnd_coef(ux, lq, c);
            const double wl = -dt * ux * K.inv_dx * lbc;
            for (int o = 0; o < 5; o++) a.cw[((size_t)16 * 5 + o) * nx + j] = wl * c[o];
            for (int i = 0; i < 16; i++) {
                const double v = a.vx[i];
                if (v == 0.0) continue;
                double qv[5];
                for (int o = -2; o <= 2; o++) qv[o + 2] = a.f[i * K.plane + bmap(j + o, nx, K.bc_x)];
                nnd_coef(v, qv, c);
                const double w = -dt * v * K.inv_dx * a.fb1[i * nx + j];
                for (int o = 0; o < 5; o++) a.cw[((size_t)i * 5 + o) * nx + j] = w * c[o];
            }
        }

        // ---- reverse sweep ----
        double Wb[16], Omb[16];
        for (int i = 0; i < 16; i++) Wb[i] = dt * a.fb1[i * nx + j];
        inverse_moments_t(K, Wb, Omb); // Omega_b = M^-T W_b (block form)
        double crb = 0.0, dqb[16], Db[16];
        for (int k = 3; k < 16; k++) {
            dqb[k] = cr * Omb[k];
            crb += dq[k] * Omb[k];
        }
        for (int k = 4; k < 16; k++) {
            Db[k] = -K.S[k] * Omb[k] + a.tne_w * 2.0 * Dk[k];
            pS[k - 4] += -Dk[k] * Omb[k];
            jt += Dk[k] * Dk[k];
        }
        const double A8b = Omb[7], A9b = Omb[8];
        const double dlb = K.chem * crb + lbc;
        pS[12] += dl * (2.0 / (DI * dt)) * crb; // dQ
        double rhob = 0.0, uxb = 0.0, uyb = 0.0, Tb = 0.0, lamb = lbc, gxb = 0.0, gyb = 0.0;
        if (ig) {
            lamb += dl_lam * dlb;
            const double ab = dl_a * dlb, bb = dl_b * dlb;
            pS[13] += pr * ab; // domega1
            pS[14] += pr * bb; // domega2
            const double pb = K.omega1 * ab + K.omega2 * bb;
            rhob += T * pb;
            Tb += rho * pb;
        }
        // A_hat_8 = rho T A8c X8, A_hat_9 = rho T A9c X9
        {
            rhob += T * A8c * X8 * A8b + T * A9c * X9 * A9b;
            Tb += rho * A8c * X8 * A8b + rho * A9c * X9 * A9b;
            const double A8cb = rho * T * X8 * A8b, X8b = rho * T * A8c * A8b;
            const double A9cb = rho * T * X9 * A9b, X9b = rho * T * A9c * A9b;
            const double S5 = K.S[4], S8 = K.S[7], S7 = K.S[6], S9 = K.S[8];
            pS[0] += (S8 / (S5 * S5)) * A8cb;
            pS[3] += (-1.0 / S5) * A8cb;
            pS[2] += (S9 / (S7 * S7)) * A9cb;
            pS[4] += (-1.0 / S7) * A9cb;
            uxb += 4.0 * gx * (1.0 - 1.0 / DI) * X8b + 2.0 * gy * X9b;
            gxb += 4.0 * ux * (1.0 - 1.0 / DI) * X8b - 4.0 * uy / DI * X9b;
            uyb += 2.0 * gy * X8b - 4.0 * gx / DI * X9b;
            gyb += 2.0 * uy * X8b + 2.0 * ux * X9b;
        }
        // d f_hat^eq / dT (k = 3..15), all linear in rho
        {
            const double u2 = ux * ux + uy * uy;
            double s = 0.0;
            for (int k = 3; k < 16; k++) s += dqb[k] * dq[k];
            rhob += s / rho;
            uxb += dqb[7] * rho * (DI + 2) + dqb[9] * 3 * rho + dqb[11] * rho +
                   dqb[13] * (2 * rho * ux + 2 * rho * ux * (DI + 4)) + dqb[14] * rho * uy * (DI + 4) +
                   dqb[15] * 2 * rho * ux;
            uyb += dqb[8] * rho * (DI + 2) + dqb[10] * rho + dqb[12] * 3 * rho + dqb[13] * 2 * rho * uy +
                   dqb[14] * rho * ux * (DI + 4) + dqb[15] * (2 * rho * uy + 2 * rho * uy * (DI + 4));
            Tb += (dqb[13] + dqb[15]) * 2 * rho * (DI + 2);
            (void)u2;
        }
        // f_hat^eq_k (k = 4..15) with qb = -Delta_b
        {
            const double u2 = ux * ux + uy * uy;
            const double A = (DI + 2) * T + u2, B = (DI + 4) * T + u2;
            double qb[16];
            for (int k = 4; k < 16; k++) qb[k] = -Db[k];
            double s = 0.0;
            for (int k = 4; k < 16; k++) s += qb[k] * q[k];
            rhob += s / rho;
            uxb += qb[4] * 2 * rho * ux + qb[5] * rho * uy + qb[7] * (rho * A + 2 * rho * ux * ux) +
                   qb[8] * 2 * rho * uy * ux + qb[9] * (3 * rho * T + 3 * rho * ux * ux) +
                   qb[10] * 2 * rho * ux * uy + qb[11] * (rho * T + rho * uy * uy) +
                   qb[13] * (2 * rho * T * ux + rho * (2 * ux * B + 2 * ux * ux * ux)) +
                   qb[14] * (rho * uy * B + 2 * rho * ux * ux * uy) +
                   qb[15] * (2 * rho * T * ux + 2 * rho * uy * uy * ux);
            uyb += qb[5] * rho * ux + qb[6] * 2 * rho * uy + qb[7] * 2 * rho * ux * uy +
                   qb[8] * (rho * A + 2 * rho * uy * uy) + qb[10] * (rho * T + rho * ux * ux) +
                   qb[11] * 2 * rho * ux * uy + qb[12] * (3 * rho * T + 3 * rho * uy * uy) +
                   qb[13] * (2 * rho * T * uy + 2 * rho * ux * ux * uy) +
                   qb[14] * (rho * ux * B + 2 * rho * ux * uy * uy) +
                   qb[15] * (2 * rho * T * uy + rho * (2 * uy * B + 2 * uy * uy * uy));
            Tb += qb[4] * rho + qb[6] * rho + qb[7] * rho * ux * (DI + 2) + qb[8] * rho * uy * (DI + 2) +
                  qb[9] * 3 * rho * ux + qb[10] * rho * uy + qb[11] * rho * ux + qb[12] * 3 * rho * uy +
                  qb[13] * (rho * (A + (DI + 2) * T) + rho * ux * ux * (DI + 4)) +
                  qb[14] * rho * ux * uy * (DI + 4) +
                  qb[15] * (rho * (A + (DI + 2) * T) + rho * uy * uy * (DI + 4));
        }
        // u.grad(lambda): the local derivative with respect to u_x
        uxb += -dt * K.inv_dx * lsel * lbc;
        for (int k = 0; k < 4; k++) a.mb[k * nx + j] = 0.0;
        for (int k = 4; k < 16; k++) a.mb[k * nx + j] = Db[k];
        a.loc[j] = rhob;
        a.loc[nx + j] = uxb;
        a.loc[2 * nx + j] = uyb;
        a.loc[3 * nx + j] = Tb;
        a.loc[4 * nx + j] = lamb;
        a.loc[5 * nx + j] = lbc;
        a.gb[j] = gxb;
        a.gb[nx + j] = gyb;
    }
    for (int q = 0; q < ADJ_NPAR; q++) block_add(pS[q], a.pacc + (size_t)q * gridDim.x, sred);
    block_add(jt * a.jw, a.jacc, sred);
}

__global__ void __launch_bounds__(ADJ_THREADS)
    adj_pass_b(const ModelConst<double> K, const AdjArgs a)
{
    const int nx = K.nx, bc = K.bc_x;
    const double DI = K.DI;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx; j += gridDim.x * blockDim.x) {
        // sum over the cells jp whose stencil reads j of their weighted coefficient at j:
        // inside the grid jp = j - o reads j at offset o; near the ends every pair is tested
        const bool inner = j >= 2 && j < nx - 2;
        auto gather = [&](const double* cwp) {
            double g = 0.0;
            if (inner) {
                for (int o = -2; o <= 2; o++) g += cwp[(size_t)(o + 2) * nx + (j - o)];
            } else {
                for (int d = -2; d <= 2; d++) {
                    const int jp = neighbour(j, d, nx, bc);
                    if (jp < 0) continue;
                    for (int o = -2; o <= 2; o++)
                        if (bmap(jp + o, nx, bc) == j) g += cwp[(size_t)(o + 2) * nx + jp];
                }
            }
            return g;
        };
        // velocity gradients of the neighbours that read u_j
        double uxb = a.loc[nx + j], uyb = a.loc[2 * nx + j];
        for (int d = -1; d <= 1; d++) {
            const int jp = neighbour(j, d, nx, bc);
            if (jp < 0) continue;
            if (bmap(jp + 1, nx, bc) == j) uxb += K.half_inv_dx * a.gb[jp], uyb += K.half_inv_dx * a.gb[nx + jp];
            if (bmap(jp - 1, nx, bc) == j) uxb -= K.half_inv_dx * a.gb[jp], uyb -= K.half_inv_dx * a.gb[nx + jp];
        }
        // macro chain: rho = m0, u = m1/rho, m2/rho, T = (m3/rho - u^2)/(D+I)
        const double rho = a.mac[j], ux = a.mac[nx + j], uy = a.mac[2 * nx + j], T = a.mac[3 * nx + j];
        const double Tb = a.loc[3 * nx + j];
        double rhob = a.loc[j];
        const double r = 1.0 / rho;
        const double Eb = Tb / DI;
        uxb += -2.0 * ux * Tb / DI;
        uyb += -2.0 * uy * Tb / DI;
        const double m1 = rho * ux, m2 = rho * uy, m3 = rho * (DI * T + ux * ux + uy * uy);
        const double rb = m1 * uxb + m2 * uyb + m3 * Eb;
        rhob += -r * r * rb;
        double mb[16];
        for (int k = 4; k < 16; k++) mb[k] = a.mb[k * nx + j];
        mb[0] = rhob;
        mb[1] = r * uxb;
        mb[2] = r * uyb;
        mb[3] = r * Eb;
        // M^T mb (block form), identity and transposed NND stencils (x only)
        double mtm[16];
        forward_moments_t(K, mb, mtm);
        for (int i = 0; i < 16; i++) {
            double s = a.fb1[i * nx + j] + mtm[i];
            if (a.vx[i] != 0.0) s += gather(a.cw + (size_t)i * 5 * nx);
            a.fb0[i * nx + j] = s;
        }
        // lambda: local parts and the transposed stencil of u.grad(lambda)
        a.lb0[j] = a.loc[4 * nx + j] + gather(a.cw + (size_t)16 * 5 * nx);
    }
}

// dJ/df of the final state from J_mis = w/2 sum_x (rho - rho*)^2 dx (rho = sum_i f_i)
__global__ void __launch_bounds__(ADJ_THREADS)
    adj_seed(const ModelConst<double> K, const AdjArgs a, const double* rho_t, double w)
{
    __shared__ double sred[ADJ_THREADS / 32];
    const int nx = K.nx;
    double jm = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx; j += gridDim.x * blockDim.x) {
        double rho = 0.0;
        for (int i = 0; i < 16; i++) rho += a.f[i * K.plane + j];
        const double d = rho - rho_t[j];
        jm += 0.5 * w * d * d * K.dx_;
        for (int i = 0; i < 16; i++) a.fb0[i * nx + j] = w * d * K.dx_;
        a.lb0[j] = 0.0;
    }
    block_add(jm, a.jacc, sred);
}

// dJ/drho0 of an equilibrium start f0 = M^-1 f_hat^eq(rho0, u0, T0): f_hat^eq is
// linear in rho0, so dJ/drho0 = sum_k (M^-T fb0)_k (M f0)_k / rho0.
__global__ void __launch_bounds__(ADJ_THREADS)
    adj_rho0(const ModelConst<double> K, const AdjArgs a, double* drho0)
{
    const int nx = K.nx;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx; j += gridDim.x * blockDim.x) {
        double f[16], m[16], fb[16];
        for (int i = 0; i < 16; i++) f[i] = a.f[i * K.plane + j], fb[i] = a.fb1[i * nx + j];
        forward_moments(K, f, m);
        double qb[16];
        inverse_moments_t(K, fb, qb);
        double s = 0.0;
        for (int k = 0; k < 16; k++) s += qb[k] * m[k];
        drho0[j] = s / m[0];
    }
}

// the objective's TNE term of one state alone: w_tne dx dt sum_x sum_k Delta_k^2
__global__ void __launch_bounds__(ADJ_THREADS)
    adj_jtne(const ModelConst<double> K, const AdjArgs a)
{
    __shared__ double sred[ADJ_THREADS / 32];
    const int nx = K.nx;
    double jt = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx; j += gridDim.x * blockDim.x) {
        double f[16], m[16], q[16];
        for (int i = 0; i < 16; i++) f[i] = a.f[i * K.plane + j];
        double rho, ux, uy, T; // as the macros kernel forms them for the reverse sweep
        recover_f64(K.cd, K.wd, K.inv_DId, f, rho, ux, uy, T);
        forward_moments(K, f, m);
        feq_moments(K.DI, rho, ux, uy, T, q);
        for (int k = 4; k < 16; k++) {
            const double D = m[k] - q[k];
            jt += D * D;
        }
    }
    block_add(jt * a.jw, a.jacc, sred);
}

// an FP32 checkpoint widened to FP64, element by element (exact)
__global__ void adj_widen(const float* __restrict__ in, double* __restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

} // namespace

int adj_grid(int nx)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (nx + ADJ_THREADS - 1) / ADJ_THREADS;
    const int cap = sms * 4;
    return need < cap ? need : cap;
}

cudaError_t launch_adj_step(const ModelConst<double>& K, const AdjArgs& a, int grid, cudaStream_t s)
{
    adj_pass_a<<<grid, ADJ_THREADS, 0, s>>>(K, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_pass_b<<<grid, ADJ_THREADS, 0, s>>>(K, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_seed(const ModelConst<double>& K, const AdjArgs& a, const double* rho_t,
                            double w, int grid, cudaStream_t s)
{
    adj_seed<<<grid, ADJ_THREADS, 0, s>>>(K, a, rho_t, w);
    return cudaGetLastError();
}

cudaError_t launch_adj_jtne(const ModelConst<double>& K, const AdjArgs& a, int grid, cudaStream_t s)
{
    adj_jtne<<<grid, ADJ_THREADS, 0, s>>>(K, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_widen(const float* in, double* out, size_t n, int grid, cudaStream_t s)
{
    adj_widen<<<grid, ADJ_THREADS, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_adj_rho0(const ModelConst<double>& K, const AdjArgs& a, double* drho0,
                            int grid, cudaStream_t s)
{
    adj_rho0<<<grid, ADJ_THREADS, 0, s>>>(K, a, drho0);
    return cudaGetLastError();
}

} // namespace lbk
