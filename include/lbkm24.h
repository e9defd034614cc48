/*
 * lbkm24.h -- C ABI of the paper's own 24-velocity model (D2V24) of the
 * multiple-relaxation-time lattice Boltzmann kinetic model for combustion of
 * Xu, Lin, Zhang and Li (arXiv:1411.6697), on GB300 (sm_103a).
 *
 * Velocities (Sec. II, Eqs. (25)-(27)): three groups of eight, each an axis
 * orbit cyc(+-1, 0) followed by a diagonal orbit (+-1, +-1), scaled by the
 * group's speed v_a, v_b, v_c and carrying eta_a, eta_b, eta_c. Order inside an
 * orbit: (1,0),(0,1),(-1,0),(0,-1) and (1,1),(-1,1),(-1,-1),(1,-1).
 *
 * One time step updates, in every cell, the 24 distribution functions f_i and
 * the reaction progress lambda:
 *   - moments f_hat = M f with all 24 rows m_1..m_24 listed after Eq. (16);
 *     rho, u, T from f_hat_1..4 (Eqs. (5)-(7)), formed in FP64;
 *   - f_hat^eq_1..24 in closed form (the same list; f_hat^eq_14 and f_hat^eq_16
 *     carry the factor T of Eq. (11));
 *   - Omega = M^-1 [-R_hat (f_hat - f_hat^eq) + A_hat] + C, with A_hat_8, A_hat_9
 *     of Eqs. (3)-(4) (sign as in the Chapman-Enskog form Eq. (29)) and the
 *     chemical term taken literally in velocity space, Eq. (24):
 *       C_i = f_i^eq Q [-(1+D) I T + I (v_i - u)^2 + eta_i^2] / (I (D+I) T^2) lambda',
 *     f^eq = M^-1 f_hat^eq, lambda' the exact reaction increment over dt / dt;
 *   - NND differences of v_i f_i (Sec. II), forward Euler; lambda by Eq. (28)
 *     with m = n = 1 (time part exact where T > T_ig, advection by NND interface
 *     values), clamped to [0, 1];
 *   - on request, the TNE measures Delta_k = f_hat_k - f_hat^eq_k (k = 5..24) and
 *     d = sqrt(sum Delta_k^2) of the state being stepped (Sec. VI, Eqs. (90)-(91)),
 *     reduced over the grid in FP64.
 *
 * Conventions are those of lbkm.h: status codes (lbkm_status), handle-owned
 * device buffers, borrowed caller arrays, FP64 row-major [ny][nx] host fields
 * (device pointers with on_device != 0), asynchronous lbkm24_step with device
 * failures surfacing as LBKM_EUNSTABLE at the next synchronising call, and no
 * thread safety per handle.
 */
#ifndef LBKM24_H
#define LBKM24_H

#include <stddef.h>
#include <stdint.h>

#include "lbkm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LBKM24_NV 24 /* discrete velocities = moments */

typedef struct lbkm24* lbkm24_t; /* opaque, owned by the library */

typedef struct {
    int32_t nx, ny;       /* grid; ny = 1 for one-dimensional runs */
    int32_t precision;    /* lbkm_precision: LBKM_F64, or LBKM_F32 (state and bulk
                             arithmetic in FP32; rho, u, T recovered in FP64 from
                             FP64 sums of the FP32 state; TNE reductions in FP64) */
    double gamma;         /* specific-heat ratio; I = 2/(gamma-1) - D, I > 0 */
    double v[3];          /* v_a, v_b, v_c (> 0) */
    double eta[3];        /* eta_a, eta_b, eta_c (>= 0) */
    double S[24];         /* relaxation rates R_1..R_24 (R_1..R_4 accepted, unused);
                             require dt * max(S_5..S_24) < 2 */
    double Q;             /* heat release per unit mass (Eq. (18)) */
    double omega1, omega2; /* Cochran rate constants of Eq. (28), m = n = 1 */
    double T_ig;          /* reaction only where T > T_ig; finite, >= 0 */
    double dx, dy, dt;    /* grid spacing and time step */
    int32_t bc_x, bc_y;   /* LBKM_BC_PERIODIC, LBKM_BC_ZERO_GRADIENT, or LBKM_BC_SIDES
                             (each side of that direction by side_bc below) */
    int32_t tne_every;    /* 0: no on-the-fly TNE; k > 0: every k-th step */
    int32_t tne_capacity; /* records kept in the device history ring (>= 1) */
    int32_t collision;    /* 0: when R_5..R_24 are all equal and tne_every = 0, step with
                             the single-relaxation-time form of Sec. V, -R (f_i -
                             [M^-1 f_hat^eq]_i) + C_i, which skips M f (the same update
                             up to rounding: A_hat vanishes for equal rates); 1: always
                             the general moment-space form */
    int32_t side_bc[4];   /* with LBKM_BC_SIDES, the sides x = 0, x = nx, y = 0, y = ny:
                             LBKM_BC_ZERO_GRADIENT (outflow), LBKM_BC_DIRICHLET (both
                             ghost layers hold the equilibrium of side_rho/ux/uy/T and
                             lambda side_lam: the fixed states of Sec. IV.C), or
                             LBKM_BC_SPECULAR (y sides: the mirror cell across the face
                             with v_y reversed, the reflecting surface of Sec. IV.C), or
                             LBKM_BC_WALL (y sides, ny >= 2: both ghost rows take the edge
                             row's f plus M^-1 [f_hat^eq(rho, u_w, T_w) - f_hat^eq(rho, u,
                             T)], rho, u, T of the edge cell, u_w = (side_ux, side_uy) and
                             T_w = side_T the wall's: non-equilibrium extrapolation,
                             Sec. IV.D; lambda copied) */
    double side_rho[4], side_ux[4], side_uy[4], side_T[4], side_lam[4]; /* Dirichlet
                             states: rho > 0, T > 0, lambda in [0, 1] */
} lbkm24_params;

/* Grid-wide TNE measures of one state (Sec. VI): index k-1 holds Delta_k;
 * Delta_1..Delta_4 are 0. Sums weighted by dx*dy, min and max unweighted. */
typedef struct {
    double sum[24], abs_sum[24], min[24], max[24];
    double d_sum, d2_sum; /* sum of d and of d^2 */
    int64_t step;         /* step index of the state the record describes */
} lbkm24_tne_global;

/* Defaults: the steady-detonation set of Sec. IV.A -- v = (2.7, 2.2, 1.2),
 * eta = (5, 3, 1.1), gamma 1.4 (I = 3), S_5..S_7 = 1e4 and the others 1e5,
 * Q = 1, T_ig = 1.1, dx = dy = 2e-4, dt = 5e-6, zero-gradient x, periodic y,
 * LBKM_F64, TNE off, tne_capacity 1; omega1 = omega2 = 0 and nx = ny = 0 must
 * be filled in. */
void lbkm24_default_params(lbkm24_params* p);

/* Validate p, build the 24x24 M, invert it (LU with partial pivoting and one
 * refinement step in long double) and allocate the two device copies of the
 * state [25][ny][pitch] (f_1..f_24, lambda). cuda_stream: a cudaStream_t on the
 * current device (NULL = legacy default stream).
 * Errors: LBKM_EINVAL (message names the field), LBKM_ESINGULAR, LBKM_ENOMEM,
 * LBKM_ECUDA; on error *out is NULL and lbkm24_last_error(NULL) has the message. */
lbkm_status lbkm24_create(const lbkm24_params* p, void* cuda_stream, lbkm24_t* out);

/* Release every resource of h (NULL is ignored), after its stream is idle. */
void lbkm24_destroy(lbkm24_t h);

/* Equilibrium start f = M^-1 f_hat^eq(rho, u, T) (Eq. (16)) and lambda (NULL: 0).
 * Resets the step counter and the TNE history. Errors: LBKM_EINVAL, LBKM_ECUDA. */
lbkm_status lbkm24_init_fields(lbkm24_t h, const double* rho, const double* ux,
                               const double* uy, const double* T, const double* lambda,
                               int on_device);

/* Advance n >= 0 steps, asynchronously; each step is one fused kernel (plus a
 * small finishing kernel on steps that reduce TNE); chunks of steps replay a
 * CUDA graph. Errors: LBKM_ESTATE, LBKM_EINVAL, LBKM_ECUDA. */
lbkm_status lbkm24_step(lbkm24_t h, int64_t n);

/* Wait for the handle's stream and check the device status word.
 * Errors: LBKM_EUNSTABLE, LBKM_ECUDA. */
lbkm_status lbkm24_sync(lbkm24_t h);

/* Steps taken since lbkm24_init_fields / lbkm24_set_state (-1 for NULL). */
int64_t lbkm24_steps_taken(lbkm24_t h);

/* rho, u_x, u_y, T, p = rho T and lambda of the current state, each [ny][nx]
 * FP64 (host or device); NULL pointers are skipped. Synchronises. */
lbkm_status lbkm24_macros(lbkm24_t h, double* rho, double* ux, double* uy, double* T,
                          double* p, double* lambda, int on_device);

/* TNE of the current state: delta, if not NULL, receives Delta_1..Delta_24 as
 * [24][ny][nx] FP64 (Delta_1..4 = 0); g, if not NULL, the grid-wide record
 * (host memory). Synchronises. */
lbkm_status lbkm24_tne(lbkm24_t h, double* delta, lbkm24_tne_global* g, int on_device);

/* Copy up to max_records on-the-fly TNE records, oldest first, to out (host);
 * *n_out receives the count. Synchronises. */
lbkm_status lbkm24_tne_history(lbkm24_t h, lbkm24_tne_global* out, int32_t max_records,
                               int32_t* n_out);

/* Bytes of one state snapshot: 25 planes of nx*ny values in the handle's
 * precision (f_1..f_24, lambda), then the int64 step counter. */
size_t lbkm24_state_bytes(lbkm24_t h);

/* Checkpoint / resume (lbkm24_state_bytes() bytes, host or device). */
lbkm_status lbkm24_get_state(lbkm24_t h, void* dst, int on_device);
lbkm_status lbkm24_set_state(lbkm24_t h, const void* src, int on_device);

/* Message of the last failing call on h (h = NULL: of the last failed create). */
const char* lbkm24_last_error(lbkm24_t h);

#ifdef __cplusplus
}
#endif

#endif /* LBKM24_H */
