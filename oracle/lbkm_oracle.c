/*
 * lbkm_oracle.c -- plain, slow, FP64 CPU oracle of the two-dimensional
 * multiple-relaxation-time lattice Boltzmann kinetic model (MRT-LBKM) for
 * combustion of Xu, Lin, Zhang and Li ("Multiple-relaxation-time lattice
 * Boltzmann kinetic model for combustion", arXiv:1411.6697).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only code allowed to load this
 * library. It shares no source, header, table or helper with the CUDA library
 * and must never sit on the product path.
 *
 * What one step computes, in the paper's order (Sec. II):
 *   1. ghost cells (2 per side) from the boundary condition: periodic, zero
 *      gradient, Dirichlet (the equilibrium of a given state, Sec. IV.C), specular
 *      reflection (Sec. IV.C, the mirror cell with v_y reversed), or a wall in y
 *      by non-equilibrium extrapolation (Sec. IV.D:
 *      ghost f = f of the adjacent fluid cell + M^-1 [f_hat^eq(rho, u_w, T_w) -
 *      f_hat^eq(rho, u, T)], rho, u, T those of the fluid cell, u_w and T_w the
 *      wall's; lambda copied);
 *   2. moments f_hat = M f and macros rho, u, T, p for every cell and ghost
 *      (Eqs. (5)-(7), the rows m_1..m_16 listed after Eq. (16));
 *   3. grad u by second-order central differences (needed by Eqs. (3)-(4));
 *   4. f_hat^eq (list after Eq. (16); entries 14 and 16 from Eq. (11)),
 *      Delta_k = f_hat_k - f_hat^eq_k (Eq. (90)), A_hat_8, A_hat_9 (Eqs. (3)-(4));
 *   5. reaction: Eq. (28) with m = n = 1, its time part integrated exactly over
 *      dt with p and T frozen at t_n, only where T > T_ig;
 *   6. chemical term in moment space C_hat_k = (d f_hat^eq_k / dT) dT/dt|_C,
 *      dT/dt|_C = 2 Q lambda' / (D + I)   (Eqs. (19)-(23));
 *   7. Omega_hat = -R_hat (f_hat - f_hat^eq) + A_hat + C_hat (sign of A as in
 *      the Chapman-Enskog form Eq. (29)); Omega = M^-1 Omega_hat;
 *   8. NND flux differences of v_i f_i (Sec. II, NND scheme of Zhang 1988);
 *   9. u . grad(lambda) with NND interface values of lambda (Eq. (28));
 *  10. forward Euler: f^{n+1} = f^n + dt (-div(v f) + Omega),
 *      lambda^{n+1} = clamp(lambda^n - dt u.grad(lambda) + dlambda_chem, 0, 1);
 *      optionally (time_scheme 1) two such steps E averaged with the state at t_n,
 *      u^{n+1} = (u^n + E(E(u^n))) / 2, the two-stage SSP Runge-Kutta scheme, or
 *      (time_scheme 2) the three-stage one, u1 = E(u^n), u2 = 3/4 u^n + 1/4 E(u1),
 *      u^{n+1} = 1/3 u^n + 2/3 E(u2) (Shu and Osher's third-order form).
 * TNE measures (Sec. VI, Eqs. (90)-(91)) are evaluated on a given state.
 *
 * The same source builds two oracles. NV = 16 (default): the 16-velocity model in
 * four orbits, chemical term in moment space as above. NV = 24 (-DNV=24): the
 * paper's own D2V24 model (Eqs. (25)-(27): three groups of an axis and a diagonal
 * orbit with speeds v_a, v_b, v_c and eta_a, eta_b, eta_c), all 24 rows m_1..m_24 of
 * M and f_hat^eq_1..24 as listed after Eq. (16), and the chemical term taken
 * literally in velocity space, Eq. (24):
 *   C_i = f_i^eq Q [-(1+D) I T + I (v_i - u)^2 + eta_i^2] / (I (D+I) T^2) lambda',
 * with f^eq = M^-1 f_hat^eq; step 7 becomes Omega = M^-1(-R_hat Delta + A_hat) + C.
 *
 * Every reading taken where the paper is silent or inconsistent (sign of A,
 * the factor T in f_hat^eq_14/16, the integrator, the NND formula, ghost cells,
 * minmod tie-break) is listed in the design notes of the repository.
 *
 * Arrays: f is [NV][ny][nx] (plane per velocity, row-major), lambda and the
 * macro fields are [ny][nx]. All FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef NV
#define NV 16 /* number of discrete velocities and of moments: 16 or 24 */
#endif
#if NV != 16 && NV != 24
#error "NV must be 16 or 24"
#endif
#define DIM 2 /* D, the spatial dimension */
#define GH 2  /* ghost cells per side */

typedef struct {
    int32_t nx, ny;
    int32_t bc_x, bc_y; /* 0 = periodic, 1 = zero gradient (copy edge cell), 2 = wall (y) */
    double vx[NV], vy[NV], eta[NV];
    double I;     /* extra (internal) degrees of freedom */
    double S[NV]; /* relaxation rates R_1..R_16 */
    double Q, omega1, omega2, T_ig;
    double dx, dy, dt;
    double wall_ux[2], wall_uy[2], wall_T[2]; /* bc_y = 2: [0] wall below y = 0, [1] above */
    /* bc_x or bc_y = 5: each side of that direction has its own condition, side_bc[s]
     * for the sides x = 0, x = nx, y = 0, y = ny: 1 zero gradient, 2 wall by
     * non-equilibrium extrapolation (y sides, wall_* [s - 2]), 3 Dirichlet (the
     * equilibrium of side_rho/ux/uy/T, lambda side_lam), 4 specular reflection (y sides:
     * the mirror cell with v_y reversed) */
    int32_t side_bc[4];
    double side_rho[4], side_ux[4], side_uy[4], side_T[4], side_lam[4];
    /* 0: forward Euler; 1: the two-stage strong-stability-preserving Runge-Kutta
     * scheme built from that step E: u1 = E(u), u^{n+1} = (u + E(u1)) / 2; 2: the
     * three-stage one, u2 = 3/4 u + 1/4 E(u1), u^{n+1} = 1/3 u + 2/3 E(u2) */
    int32_t time_scheme;
} orc_params;

/* number of doubles in one TNE global record */
#define ORC_TNE_LEN (4 * NV + 2)

/* ------------------------------------------------------------------ */
/* Matrix M: rows m_1..m_NV of Sec. II (list after Eq. (16)).         */
/* ------------------------------------------------------------------ */
void orc_build_M(const orc_params* p, double* M /* [NV][NV] */)
{
    for (int i = 0; i < NV; i++) {
        double vx = p->vx[i], vy = p->vy[i];
        double w = vx * vx + vy * vy + p->eta[i] * p->eta[i]; /* v^2 + eta^2 */
#if NV == 24
        double e2 = p->eta[i] * p->eta[i], v2 = vx * vx + vy * vy;
#endif
        double col[NV] = {
            1.0,             /* m1  */
            vx,              /* m2  */
            vy,              /* m3  */
            w,               /* m4  */
            vx * vx,         /* m5  */
            vx * vy,         /* m6  */
            vy * vy,         /* m7  */
            w * vx,          /* m8  */
            w * vy,          /* m9  */
            vx * vx * vx,    /* m10 */
            vx * vx * vy,    /* m11 */
            vx * vy * vy,    /* m12 */
            vy * vy * vy,    /* m13 */
            w * vx * vx,     /* m14 */
            w * vx * vy,     /* m15 */
            w * vy * vy,     /* m16 */
#if NV == 24
            e2 * vx * vx,    /* m17 */
            e2 * vx * vy,    /* m18 */
            e2 * vy * vy,    /* m19 */
            w * e2,          /* m20 */
            w * v2 * vx,     /* m21 */
            w * v2 * vy,     /* m22 */
            w * e2 * vx,     /* m23 */
            w * e2 * vy,     /* m24 */
#endif
        };
        for (int k = 0; k < NV; k++) M[k * NV + i] = col[k];
    }
}

/* Gauss-Jordan inversion with partial pivoting in long double.
 * Returns 0 on success, -1 if a pivot vanishes (singular M). The paper fixes
 * M^-1 numerically before the main loop (Sec. II, Sec. V). */
int orc_invert(const double* M, double* Minv)
{
    long double a[NV][2 * NV];
    for (int r = 0; r < NV; r++)
        for (int c = 0; c < 2 * NV; c++)
            a[r][c] = (c < NV) ? (long double)M[r * NV + c] : (long double)((c - NV) == r);
    long double scale = 0;
    for (int r = 0; r < NV; r++)
        for (int c = 0; c < NV; c++)
            if (fabsl(a[r][c]) > scale) scale = fabsl(a[r][c]);
    for (int col = 0; col < NV; col++) {
        int piv = col;
        for (int r = col + 1; r < NV; r++)
            if (fabsl(a[r][col]) > fabsl(a[piv][col])) piv = r;
        if (fabsl(a[piv][col]) <= 1e-14L * scale) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * NV; c++) {
                long double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        long double d = a[col][col];
        for (int c = 0; c < 2 * NV; c++) a[col][c] /= d;
        for (int r = 0; r < NV; r++) {
            if (r == col) continue;
            long double m = a[r][col];
            if (m == 0) continue;
            for (int c = 0; c < 2 * NV; c++) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < NV; r++)
        for (int c = 0; c < NV; c++) Minv[r * NV + c] = (double)a[r][NV + c];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Equilibrium moments and their temperature derivative.              */
/* ------------------------------------------------------------------ */

/* f_hat^eq_1..16 (Sec. II, list after Eq. (16)). Entries 14 and 16 follow the
 * moment relation Eq. (11), which carries a factor T on the first term. */
void orc_feq_moments(double rho, double ux, double uy, double T, double I, double* out)
{
    const double D = DIM;
    double u2 = ux * ux + uy * uy;
    double A = (D + I + 2.0) * T + u2;
    double B = (D + I + 4.0) * T + u2;
    out[0] = rho;
    out[1] = rho * ux;
    out[2] = rho * uy;
    out[3] = rho * ((D + I) * T + u2);
    out[4] = rho * (T + ux * ux);
    out[5] = rho * ux * uy;
    out[6] = rho * (T + uy * uy);
    out[7] = rho * ux * A;
    out[8] = rho * uy * A;
    out[9] = 3.0 * rho * ux * T + rho * ux * ux * ux;
    out[10] = rho * uy * T + rho * ux * ux * uy;
    out[11] = rho * ux * T + rho * ux * uy * uy;
    out[12] = 3.0 * rho * uy * T + rho * uy * uy * uy;
    out[13] = rho * A * T + rho * ux * ux * B;
    out[14] = rho * ux * uy * B;
    out[15] = rho * A * T + rho * uy * uy * B;
#if NV == 24
    /* f_hat^eq_17..24, the same list (moment relations Eqs. (12)-(15)) */
    const double IT = I * T;
    const double C = u2 * u2 + (D + 2.0) * (D + I + 4.0) * T * T + (2.0 * D + I + 8.0) * u2 * T;
    out[16] = rho * IT * T + rho * ux * ux * IT;
    out[17] = rho * ux * uy * IT;
    out[18] = rho * IT * T + rho * uy * uy * IT;
    out[19] = rho * IT * (u2 + (D + 3.0 * I) * T);
    out[20] = rho * ux * C;
    out[21] = rho * uy * C;
    out[22] = rho * ux * IT * (u2 + (D + 3.0 * I + 2.0) * T);
    out[23] = rho * uy * IT * (u2 + (D + 3.0 * I + 2.0) * T);
#endif
}

/* d f_hat^eq_k / dT at fixed rho and u (the chemical term keeps rho and u
 * unchanged, Eq. (20)). */
void orc_dfeq_dT(double rho, double ux, double uy, double T, double I, double* out)
{
    const double D = DIM;
    double u2 = ux * ux + uy * uy;
    double dAT = 2.0 * (D + I + 2.0) * T + u2; /* d(A T)/dT */
    out[0] = 0.0;
    out[1] = 0.0;
    out[2] = 0.0;
    out[3] = rho * (D + I);
    out[4] = rho;
    out[5] = 0.0;
    out[6] = rho;
    out[7] = rho * ux * (D + I + 2.0);
    out[8] = rho * uy * (D + I + 2.0);
    out[9] = 3.0 * rho * ux;
    out[10] = rho * uy;
    out[11] = rho * ux;
    out[12] = 3.0 * rho * uy;
    out[13] = rho * dAT + rho * ux * ux * (D + I + 4.0);
    out[14] = rho * ux * uy * (D + I + 4.0);
    out[15] = rho * dAT + rho * uy * uy * (D + I + 4.0);
#if NV == 24
    const double dC = 2.0 * (D + 2.0) * (D + I + 4.0) * T + (2.0 * D + I + 8.0) * u2;
    out[16] = 2.0 * rho * I * T + rho * ux * ux * I;
    out[17] = rho * ux * uy * I;
    out[18] = 2.0 * rho * I * T + rho * uy * uy * I;
    out[19] = rho * I * (u2 + 2.0 * (D + 3.0 * I) * T);
    out[20] = rho * ux * dC;
    out[21] = rho * uy * dC;
    out[22] = rho * ux * I * (u2 + 2.0 * (D + 3.0 * I + 2.0) * T);
    out[23] = rho * uy * I * (u2 + 2.0 * (D + 3.0 * I + 2.0) * T);
#endif
}

/* ------------------------------------------------------------------ */
/* Small helpers                                                       */
/* ------------------------------------------------------------------ */

/* minmod limiter of the NND scheme: 0 unless a and b share a sign, else the
 * argument of smaller magnitude (a on a tie). */
static double minmod(double a, double b)
{
    int same = (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0);
    if (!same) return 0.0;
    return fabs(a) <= fabs(b) ? a : b;
}

/* NND numerical flux H_{j+1/2} of F = v f from f_{j-1}, f_j, f_{j+1}, f_{j+2}
 * with the flux split F+ = max(v,0) f, F- = min(v,0) f:
 *   H = F+_j + 1/2 mm(F+_j - F+_{j-1}, F+_{j+1} - F+_j)
 *     + F-_{j+1} - 1/2 mm(F-_{j+1} - F-_j, F-_{j+2} - F-_{j+1}). */
static double nnd_face(double v, double fm1, double f0, double fp1, double fp2)
{
    double vp = v > 0.0 ? v : 0.0;
    double vm = v < 0.0 ? v : 0.0;
    double Pm1 = vp * fm1, P0 = vp * f0, P1 = vp * fp1;
    double N0 = vm * f0, N1 = vm * fp1, N2 = vm * fp2;
    return P0 + 0.5 * minmod(P0 - Pm1, P1 - P0) + N1 - 0.5 * minmod(N1 - N0, N2 - N1);
}

/* Left and right NND interface values of a scalar at j+1/2. */
static double nnd_left(double qm1, double q0, double qp1)
{
    return q0 + 0.5 * minmod(q0 - qm1, qp1 - q0);
}
static double nnd_right(double q0, double qp1, double qp2)
{
    return qp1 - 0.5 * minmod(qp1 - q0, qp2 - qp1);
}

static int map_index(int j, int n, int bc)
{
    if (bc == 0) {
        j %= n;
        if (j < 0) j += n;
        return j;
    }
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

static void macros_of(const double* fh, double I, double* rho, double* ux, double* uy, double* T)
{
    /* Eqs. (5)-(7): rho = f_hat_1, rho u = f_hat_2,3, rho[(D+I)T + u^2] = f_hat_4 */
    double r = fh[0];
    double x = fh[1] / r, y = fh[2] / r;
    *rho = r;
    *ux = x;
    *uy = y;
    *T = (fh[3] / r - (x * x + y * y)) / (DIM + I);
}

/* Exact increment of lambda over dt from d(lambda)/dt = (1-lambda)(a + b lambda),
 * a = omega1 p, b = omega2 p (Eq. (28), m = n = 1, spatial part excluded). */
double orc_reaction_increment(double lam, double a, double b, double dt)
{
    double mu0 = 1.0 - lam;
    if (b == 0.0) return mu0 * (-expm1(-a * dt));
    double k = a + b;
    double e = exp(-k * dt);
    double mu = k * mu0 * e / (k - b * mu0 * (1.0 - e));
    return mu0 - mu;
}

/* ------------------------------------------------------------------ */
/* Initialisation, macros, TNE                                         */
/* ------------------------------------------------------------------ */

/* f_i = sum_k Minv[i][k] f_hat^eq_k(rho, u, T) for every cell (Eq. (16)). */
void orc_init(const orc_params* p, const double* Minv, const double* rho, const double* ux,
              const double* uy, const double* T, double* f)
{
    size_t n = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < n; c++) {
        double fe[NV];
        orc_feq_moments(rho[c], ux[c], uy[c], T[c], p->I, fe);
        for (int i = 0; i < NV; i++) {
            double s = 0.0;
            for (int k = 0; k < NV; k++) s += Minv[i * NV + k] * fe[k];
            f[(size_t)i * n + c] = s;
        }
    }
}

void orc_moments_cell(const double* M, const double* f, size_t n, size_t c, double* fh)
{
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int i = 0; i < NV; i++) s += M[k * NV + i] * f[(size_t)i * n + c];
        fh[k] = s;
    }
}

/* rho, u_x, u_y, T, p for every cell; any output pointer may be NULL. */
void orc_macros(const orc_params* p, const double* M, const double* f, double* rho, double* ux,
                double* uy, double* T, double* pr)
{
    size_t n = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < n; c++) {
        double fh[NV], r, x, y, t;
        orc_moments_cell(M, f, n, c, fh);
        macros_of(fh, p->I, &r, &x, &y, &t);
        if (rho) rho[c] = r;
        if (ux) ux[c] = x;
        if (uy) uy[c] = y;
        if (T) T[c] = t;
        if (pr) pr[c] = r * t;
    }
}

/* TNE measures of a state (Sec. VI): Delta_k = f_hat_k - f_hat^eq_k (Eq. (90)),
 * Delta_1..4 = 0 exactly by conservation, d = sqrt(sum_k Delta_k^2) (Eq. (91)).
 * delta: [NV][ny][nx] or NULL. rec: ORC_TNE_LEN doubles or NULL, laid out as
 * sum[NV], abs_sum[NV], min[NV], max[NV], d_sum, d2_sum with sums weighted by
 * dx*dy (min and max unweighted). */
void orc_tne(const orc_params* p, const double* M, const double* f, double* delta, double* rec)
{
    size_t n = (size_t)p->nx * p->ny;
    double w = p->dx * p->dy;
    double sum[NV], asum[NV], mn[NV], mx[NV], dsum = 0.0, d2sum = 0.0;
    for (int k = 0; k < NV; k++) {
        sum[k] = 0.0;
        asum[k] = 0.0;
        mn[k] = INFINITY;
        mx[k] = -INFINITY;
    }
    for (size_t c = 0; c < n; c++) {
        double fh[NV], fe[NV], r, x, y, t, D[NV], d2 = 0.0;
        orc_moments_cell(M, f, n, c, fh);
        macros_of(fh, p->I, &r, &x, &y, &t);
        orc_feq_moments(r, x, y, t, p->I, fe);
        for (int k = 0; k < NV; k++) {
            D[k] = (k < 4) ? 0.0 : fh[k] - fe[k];
            d2 += D[k] * D[k];
            if (delta) delta[(size_t)k * n + c] = D[k];
            sum[k] += D[k] * w;
            asum[k] += fabs(D[k]) * w;
            if (D[k] < mn[k]) mn[k] = D[k];
            if (D[k] > mx[k]) mx[k] = D[k];
        }
        dsum += sqrt(d2) * w;
        d2sum += d2 * w;
    }
    if (rec) {
        for (int k = 0; k < NV; k++) {
            rec[k] = sum[k];
            rec[NV + k] = asum[k];
            rec[2 * NV + k] = mn[k];
            rec[3 * NV + k] = mx[k];
        }
        rec[4 * NV] = dsum;
        rec[4 * NV + 1] = d2sum;
    }
}

/* ------------------------------------------------------------------ */
/* One time step                                                        */
/* ------------------------------------------------------------------ */

/* (f, lam) at t_n -> (f_new, lam_new) at t_{n+1}. Returns 0, or -1 on
 * allocation failure. f_new/lam_new must not alias f/lam. */
int orc_step(const orc_params* p, const double* M, const double* Minv, const double* f,
             const double* lam, double* f_new, double* lam_new)
{
    const int nx = p->nx, ny = p->ny;
    const int gx = nx + 2 * GH, gy = ny + 2 * GH;
    const size_t n = (size_t)nx * ny, ng = (size_t)gx * gy;
    const double D = DIM, I = p->I;

    /* 1. ghost-extended copies of f and lambda */
    double* fg = malloc(sizeof(double) * NV * ng);
    double* lg = malloc(sizeof(double) * ng);
    /* 2. moments and macros of every extended cell */
    double* fhg = malloc(sizeof(double) * NV * ng);
    double* rg = malloc(sizeof(double) * ng);
    double* uxg = malloc(sizeof(double) * ng);
    double* uyg = malloc(sizeof(double) * ng);
    double* Tg = malloc(sizeof(double) * ng);
    if (!fg || !lg || !fhg || !rg || !uxg || !uyg || !Tg) {
        free(fg); free(lg); free(fhg); free(rg); free(uxg); free(uyg); free(Tg);
        return -1;
    }
    /* Dirichlet ghost values of each side: f = M^-1 f_hat^eq(side state) */
    double fd[4][NV];
    for (int s = 0; s < 4; s++) {
        double fe[NV];
        orc_feq_moments(p->side_rho[s], p->side_ux[s], p->side_uy[s], p->side_T[s], I, fe);
        for (int i = 0; i < NV; i++) {
            double acc = 0.0;
            for (int k = 0; k < NV; k++) acc += Minv[i * NV + k] * fe[k];
            fd[s][i] = acc;
        }
    }
    /* the velocity with v_y reversed, for specular reflection */
    int mirror[NV];
    for (int i = 0; i < NV; i++) {
        mirror[i] = i;
        for (int j = 0; j < NV; j++)
            if (p->vx[j] == p->vx[i] && p->vy[j] == -p->vy[i] && p->eta[j] == p->eta[i]) mirror[i] = j;
    }
    for (int jy = 0; jy < gy; jy++)
        for (int jx = 0; jx < gx; jx++) {
            const int x = jx - GH, y = jy - GH;
            const size_t dst = (size_t)jy * gx + jx;
            const int ys = y < 0 ? 2 : 3, xs = x < 0 ? 0 : 1;
            const int cy = (y >= 0 && y < ny) ? -1 : (p->bc_y == 5 ? p->side_bc[ys] : p->bc_y);
            const int cx = (x >= 0 && x < nx) ? -1 : (p->bc_x == 5 ? p->side_bc[xs] : p->bc_x);
            if (cy == 3 || cx == 3) { /* Dirichlet (a y side first; corners are never read) */
                const int s = cy == 3 ? ys : xs;
                for (int i = 0; i < NV; i++) fg[(size_t)i * ng + dst] = fd[s][i];
                lg[dst] = p->side_lam[s];
                continue;
            }
            int sx = cx == -1 ? x : map_index(x, nx, cx == 0 ? 0 : 1);
            int sy = cy == -1 ? y : map_index(y, ny, cy == 0 ? 0 : 1);
            int mir = 0;
            if (cy == 4) { /* specular: the mirror row across the wall face */
                sy = y < 0 ? -y - 1 : 2 * ny - 1 - y;
                mir = 1;
            }
            const size_t src = (size_t)sy * nx + sx;
            for (int i = 0; i < NV; i++)
                fg[(size_t)i * ng + dst] = f[(size_t)(mir ? mirror[i] : i) * n + src];
            lg[dst] = lam[src];
        }

    /* walls in y: non-equilibrium extrapolation into both ghost rows of each side */
    if (p->bc_y == 2 || p->bc_y == 5) {
        for (int side = 0; side < 2; side++) {
            if (p->bc_y == 5 && p->side_bc[2 + side] != 2) continue;
            const int jsrc = side == 0 ? GH : GH + ny - 1;
            for (int jx = 0; jx < gx; jx++) {
                const size_t src = (size_t)jsrc * gx + jx;
                double fh[NV], r, ux, uy, T, fw[NV], fs[NV], d[NV];
                orc_moments_cell(M, fg, ng, src, fh);
                macros_of(fh, I, &r, &ux, &uy, &T);
                orc_feq_moments(r, p->wall_ux[side], p->wall_uy[side], p->wall_T[side], I, fw);
                orc_feq_moments(r, ux, uy, T, I, fs);
                for (int i = 0; i < NV; i++) {
                    double s = 0.0;
                    for (int k = 0; k < NV; k++) s += Minv[i * NV + k] * (fw[k] - fs[k]);
                    d[i] = s;
                }
                for (int g = 0; g < GH; g++) {
                    const int jg = side == 0 ? g : GH + ny + g;
                    const size_t dst = (size_t)jg * gx + jx;
                    for (int i = 0; i < NV; i++)
                        fg[(size_t)i * ng + dst] = fg[(size_t)i * ng + src] + d[i];
                }
            }
        }
    }

#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)ng; c++) {
        double fh[NV];
        orc_moments_cell(M, fg, ng, (size_t)c, fh);
        for (int k = 0; k < NV; k++) fhg[(size_t)k * ng + c] = fh[k];
        macros_of(fh, I, &rg[c], &uxg[c], &uyg[c], &Tg[c]);
    }

#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < (long)n; cell++) {
        {
            const int x = (int)(cell % nx), y = (int)(cell / nx);
            const int jx = x + GH, jy = y + GH;
            const size_t g = (size_t)jy * gx + jx;
            const size_t out = (size_t)y * nx + x;
#define G(dxo, dyo) (g + (long)(dyo) * gx + (dxo))
            double rho = rg[g], ux = uxg[g], uy = uyg[g], T = Tg[g];
            double pr = rho * T;

            /* 3. velocity gradients, second-order central differences */
            double dux_dx = (uxg[G(1, 0)] - uxg[G(-1, 0)]) / (2.0 * p->dx);
            double duy_dx = (uyg[G(1, 0)] - uyg[G(-1, 0)]) / (2.0 * p->dx);
            double dux_dy = (uxg[G(0, 1)] - uxg[G(0, -1)]) / (2.0 * p->dy);
            double duy_dy = (uyg[G(0, 1)] - uyg[G(0, -1)]) / (2.0 * p->dy);
            double theta = dux_dx + duy_dy;

            /* 4. equilibrium moments, non-equilibrium parts, A_hat_8, A_hat_9 */
            double fh[NV], fe[NV], dfe[NV], Delta[NV];
            for (int k = 0; k < NV; k++) fh[k] = fhg[(size_t)k * ng + g];
            orc_feq_moments(rho, ux, uy, T, I, fe);
            for (int k = 0; k < NV; k++) Delta[k] = (k < 4) ? 0.0 : fh[k] - fe[k];
            double Ahat[NV];
            for (int k = 0; k < NV; k++) Ahat[k] = 0.0;
            Ahat[7] = rho * T * (p->S[4] - p->S[7]) / p->S[4] *
                      (4.0 * ux * (dux_dx - theta / (D + I)) + 2.0 * uy * (duy_dx + dux_dy));
            Ahat[8] = rho * T * (p->S[6] - p->S[8]) / p->S[6] *
                      (4.0 * uy * (duy_dy - theta / (D + I)) + 2.0 * ux * (duy_dx + dux_dy));

            /* 5. reaction over dt with p, T frozen at t_n; only above ignition */
            double lam0 = lg[g];
            double dlam_chem = 0.0;
            if (T > p->T_ig)
                dlam_chem = orc_reaction_increment(lam0, p->omega1 * pr, p->omega2 * pr, p->dt);
            double lam_rate = dlam_chem / p->dt; /* lambda' */

            double Om_hat[NV], Om[NV];
#if NV == 24
            /* 6-7. collision in moment space, back to velocity space, plus the
             * chemical term of Eq. (24) in velocity space on f^eq = M^-1 f_hat^eq */
            (void)dfe;
            for (int k = 0; k < NV; k++) Om_hat[k] = -p->S[k] * Delta[k] + Ahat[k];
            for (int i = 0; i < NV; i++) {
                double s = 0.0, fq = 0.0;
                for (int k = 0; k < NV; k++) {
                    s += Minv[i * NV + k] * Om_hat[k];
                    fq += Minv[i * NV + k] * fe[k];
                }
                const double cx = p->vx[i] - ux, cy = p->vy[i] - uy;
                const double shape = -(1.0 + D) * I * T + I * (cx * cx + cy * cy) +
                                     p->eta[i] * p->eta[i];
                Om[i] = s + fq * p->Q * shape / (I * (D + I) * T * T) * lam_rate;
            }
#else
            /* 6. chemical term in moment space */
            orc_dfeq_dT(rho, ux, uy, T, I, dfe);
            double dTdt = 2.0 * p->Q * lam_rate / (D + I);

            /* 7. collision in moment space, back to velocity space */
            for (int k = 0; k < NV; k++)
                Om_hat[k] = -p->S[k] * Delta[k] + Ahat[k] + dfe[k] * dTdt;
            for (int i = 0; i < NV; i++) {
                double s = 0.0;
                for (int k = 0; k < NV; k++) s += Minv[i * NV + k] * Om_hat[k];
                Om[i] = s;
            }
#endif

            /* 8. NND flux differences and 10. forward Euler for each f_i */
            for (int i = 0; i < NV; i++) {
                const double* fi = fg + (size_t)i * ng;
                double vx = p->vx[i], vy = p->vy[i];
                double Hxp = nnd_face(vx, fi[G(-1, 0)], fi[G(0, 0)], fi[G(1, 0)], fi[G(2, 0)]);
                double Hxm = nnd_face(vx, fi[G(-2, 0)], fi[G(-1, 0)], fi[G(0, 0)], fi[G(1, 0)]);
                double Hyp = nnd_face(vy, fi[G(0, -1)], fi[G(0, 0)], fi[G(0, 1)], fi[G(0, 2)]);
                double Hym = nnd_face(vy, fi[G(0, -2)], fi[G(0, -1)], fi[G(0, 0)], fi[G(0, 1)]);
                double adv = (Hxp - Hxm) / p->dx + (Hyp - Hym) / p->dy;
                f_new[(size_t)i * n + out] = fi[g] + p->dt * (Om[i] - adv);
            }

            /* 9. u . grad(lambda) with NND interface values, then update */
            double lLp = nnd_left(lg[G(-1, 0)], lg[G(0, 0)], lg[G(1, 0)]);
            double lLm = nnd_left(lg[G(-2, 0)], lg[G(-1, 0)], lg[G(0, 0)]);
            double lRp = nnd_right(lg[G(0, 0)], lg[G(1, 0)], lg[G(2, 0)]);
            double lRm = nnd_right(lg[G(-1, 0)], lg[G(0, 0)], lg[G(1, 0)]);
            double adv_x = (ux > 0.0 ? ux : 0.0) * (lLp - lLm) / p->dx +
                           (ux < 0.0 ? ux : 0.0) * (lRp - lRm) / p->dx;
            double bLp = nnd_left(lg[G(0, -1)], lg[G(0, 0)], lg[G(0, 1)]);
            double bLm = nnd_left(lg[G(0, -2)], lg[G(0, -1)], lg[G(0, 0)]);
            double bRp = nnd_right(lg[G(0, 0)], lg[G(0, 1)], lg[G(0, 2)]);
            double bRm = nnd_right(lg[G(0, -1)], lg[G(0, 0)], lg[G(0, 1)]);
            double adv_y = (uy > 0.0 ? uy : 0.0) * (bLp - bLm) / p->dy +
                           (uy < 0.0 ? uy : 0.0) * (bRp - bRm) / p->dy;
            double ln = lam0 - p->dt * (adv_x + adv_y) + dlam_chem;
            lam_new[out] = ln < 0.0 ? 0.0 : (ln > 1.0 ? 1.0 : ln);
#undef G
        }
    }
    free(fg); free(lg); free(fhg); free(rg); free(uxg); free(uyg); free(Tg);
    return 0;
}

/* nsteps steps in place on (f, lam). If tne is non-NULL it receives, for each
 * step s, the TNE record of the state at the start of that step
 * (nsteps * ORC_TNE_LEN doubles). Returns 0 or -1 on allocation failure. */
int orc_run(const orc_params* p, const double* M, const double* Minv, double* f, double* lam,
            int64_t nsteps, double* tne)
{
    size_t n = (size_t)p->nx * p->ny;
    double* f2 = malloc(sizeof(double) * NV * n);
    double* l2 = malloc(sizeof(double) * n);
    if (!f2 || !l2) {
        free(f2); free(l2);
        return -1;
    }
    double *fa = f, *la = lam, *fb = f2, *lb = l2;
    double *f3 = NULL, *l3 = NULL;
    if (p->time_scheme == 1 || p->time_scheme == 2) {
        f3 = malloc(sizeof(double) * NV * n);
        l3 = malloc(sizeof(double) * n);
        if (!f3 || !l3) {
            free(f2); free(l2); free(f3); free(l3);
            return -1;
        }
    }
    for (int64_t s = 0; s < nsteps; s++) {
        if (tne) orc_tne(p, M, fa, NULL, tne + (size_t)s * ORC_TNE_LEN);
        if (orc_step(p, M, Minv, fa, la, fb, lb) != 0) {
            free(f2); free(l2); free(f3); free(l3);
            return -1;
        }
        if (p->time_scheme == 1) { /* second stage from u1, then the average with u^n */
            if (orc_step(p, M, Minv, fb, lb, f3, l3) != 0) {
                free(f2); free(l2); free(f3); free(l3);
                return -1;
            }
            for (size_t i = 0; i < NV * n; i++) fb[i] = 0.5 * (fa[i] + f3[i]);
            for (size_t i = 0; i < n; i++) lb[i] = 0.5 * (la[i] + l3[i]);
        } else if (p->time_scheme == 2) {
            /* three stages: u2 = 3/4 u + 1/4 E(u1), u^{n+1} = 1/3 u + 2/3 E(u2) */
            if (orc_step(p, M, Minv, fb, lb, f3, l3) != 0) {
                free(f2); free(l2); free(f3); free(l3);
                return -1;
            }
            for (size_t i = 0; i < NV * n; i++) f3[i] = 0.75 * fa[i] + 0.25 * f3[i];
            for (size_t i = 0; i < n; i++) l3[i] = 0.75 * la[i] + 0.25 * l3[i];
            if (orc_step(p, M, Minv, f3, l3, fb, lb) != 0) {
                free(f2); free(l2); free(f3); free(l3);
                return -1;
            }
            for (size_t i = 0; i < NV * n; i++) fb[i] = fa[i] / 3.0 + 2.0 * fb[i] / 3.0;
            for (size_t i = 0; i < n; i++) lb[i] = la[i] / 3.0 + 2.0 * lb[i] / 3.0;
        }
        double* t = fa; fa = fb; fb = t;
        t = la; la = lb; lb = t;
    }
    free(f3); free(l3);
    if (fa != f) {
        memcpy(f, fa, sizeof(double) * NV * n);
        memcpy(lam, la, sizeof(double) * n);
    }
    free(f2); free(l2);
    return 0;
}

/* One forward-Euler step of pure linear advection d(q)/dt + v d(q)/dx = 0 on a
 * 1-D grid of n cells with the same NND flux as the kinetic step (used to pin
 * the scheme on its own: conservation, no new extrema, order of accuracy). */
void orc_nnd_advect_1d(double v, const double* q, double* q_new, int32_t n, int32_t bc, double dt,
                       double dx)
{
    for (int j = 0; j < n; j++) {
        double a[5];
        for (int o = -2; o <= 2; o++) a[o + 2] = q[map_index(j + o, n, bc)];
        double Hp = nnd_face(v, a[1], a[2], a[3], a[4]);
        double Hm = nnd_face(v, a[0], a[1], a[2], a[3]);
        q_new[j] = q[j] - dt * (Hp - Hm) / dx;
    }
}
