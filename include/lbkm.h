/*
 * lbkm.h -- C ABI of the GB300 (sm_103a) implementation of the two-dimensional
 * multiple-relaxation-time lattice Boltzmann kinetic model for combustion of
 * Xu, Lin, Zhang and Li (arXiv:1411.6697).
 *
 * One time step updates, in every cell, the 16 discrete distribution functions
 * f_i and the reaction progress lambda:
 *   - moments f_hat = M f, macros rho, u, T (Sec. II, Eqs. (5)-(7), rows m_1..m_16
 *     of M listed after Eq. (16));
 *   - analytic equilibrium moments f_hat^eq (list after Eq. (16); f_hat^eq_14 and
 *     f_hat^eq_16 carry the factor T of Eq. (11));
 *   - relaxation in moment space with the diagonal rates R_k (= S_k here), the
 *     modification terms A_hat_8, A_hat_9 (Eqs. (3)-(4), sign as in the
 *     Chapman-Enskog form Eq. (29)) and the chemical term
 *     C_hat_k = (d f_hat^eq_k/dT) dT/dt|_C, dT/dt|_C = 2 Q lambda'/(D+I)
 *     (Eqs. (19)-(23));
 *   - back-transform Omega = M^-1 Omega_hat (M^-1 fixed before the main loop,
 *     Sec. II and Sec. V);
 *   - NND finite differences of v_i f_i in space (Sec. II) and forward Euler in
 *     time; lambda follows Eq. (28) with m = n = 1, its time part integrated
 *     exactly over dt where T > T_ig and its advection by NND interface values;
 *   - on request, the thermodynamic non-equilibrium (TNE) measures of the state
 *     being stepped, Delta_k = f_hat_k - f_hat^eq_k and d = sqrt(sum Delta_k^2)
 *     (Sec. VI, Eqs. (90)-(91)), reduced over the grid on the fly.
 *
 * Velocity model: 16 velocities in four orbits of four (kind 0 = axis set
 * cyc(+-1, 0), kind 1 = diagonal set (+-1, +-1)), each orbit with its own speed
 * and eta: the D2V24 construction of Sec. II (Eqs. (25)-(27)) reduced to the 16
 * velocities that Sec. VII allows. A non-singular 16x16 M needs exactly two
 * orbits of each kind; the library takes them in the order axis, diagonal,
 * axis, diagonal. Velocities inside an orbit: (1,0),(0,1),(-1,0),(0,-1) and
 * (1,1),(-1,1),(-1,-1),(1,-1), times the orbit speed.
 *
 * Conventions
 *   - Every call returns an lbkm_status; nothing is thrown across the ABI.
 *     lbkm_last_error() gives a message for the last failing call on a handle.
 *   - The handle owns its device buffers. Caller arrays are borrowed for the
 *     duration of a call only.
 *   - Host field arrays are FP64, row-major [ny][nx]. With on_device != 0 the
 *     pointers are device pointers (FP64, same layout) on the handle's device.
 *   - lbkm_step() is asynchronous on the handle's stream; device-side failures
 *     (non-finite or non-positive rho or T) surface as LBKM_EUNSTABLE at the
 *     next synchronising call (lbkm_macros, lbkm_tne, lbkm_sync, ...).
 *   - Calls on one handle are not thread-safe. Different handles are
 *     independent.
 */
#ifndef LBKM_H
#define LBKM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBKM_NV 16 /* discrete velocities = moments */

typedef struct lbkm* lbkm_t; /* opaque, owned by the library */

typedef enum {
    LBKM_OK = 0,
    LBKM_EINVAL = 1,    /* bad argument or parameter set */
    LBKM_ENOMEM = 2,    /* device or host allocation failed */
    LBKM_ECUDA = 3,     /* CUDA runtime error (message in lbkm_last_error) */
    LBKM_ESINGULAR = 4, /* the velocity set gives a singular M */
    LBKM_EUNSTABLE = 5, /* a cell reached non-finite or non-positive rho or T */
    LBKM_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
    LBKM_ESTATE = 7     /* call out of order (e.g. step before init_fields) */
} lbkm_status;

typedef enum {
    LBKM_F64 = 0, /* plain form: state and all arithmetic in FP64 */
    LBKM_F32 = 1  /* state and bulk arithmetic in FP32; conserved-moment
                     recovery and TNE reductions as set by lbkm_recovery */
} lbkm_precision;

typedef enum {
    LBKM_RECOVER_F64 = 0,  /* rho, u, T formed in FP64 from the conserved moments
                              rho, rho u, rho[(D+I)T+u^2]; on 2-D grids those sums
                              are first taken exactly (error-free FP32 transforms)
                              and carried into FP64 as hi + lo */
    LBKM_RECOVER_DF32 = 1  /* same quantities in double-float (pairs of FP32 with
                              error-free transforms), ~48-bit significand, run on
                              the FP32 pipes */
} lbkm_recovery;

/* LBKM_BC_WALL (bc_y only, ny >= 2, 2-D grids): walls below row 0 and above row ny-1
 * by non-equilibrium extrapolation (Sec. IV.D): each ghost cell takes the f of the
 * adjacent fluid cell plus M^-1 [f_hat^eq(rho, u_w, T_w) - f_hat^eq(rho, u, T)], with
 * rho, u, T those of the fluid cell and u_w, T_w the wall's (wall_ux/uy/T below);
 * lambda is copied from the fluid cell. */
/* LBKM_BC_SIDES (bc_x or bc_y): the two sides of that direction take their own
 * conditions from side_bc[] (x = 0, x = nx, y = 0, y = ny): LBKM_BC_ZERO_GRADIENT,
 * LBKM_BC_WALL (y sides), LBKM_BC_DIRICHLET (ghost cells hold the equilibrium of
 * side_rho/ux/uy/T and lambda side_lam: the fixed inflow states of Sec. IV.C) or
 * LBKM_BC_SPECULAR (y sides: the ghost cell mirrors the fluid cell across the face with
 * v_y reversed, the reflecting surface of Sec. IV.C). */
typedef enum {
    LBKM_BC_PERIODIC = 0,
    LBKM_BC_ZERO_GRADIENT = 1,
    LBKM_BC_WALL = 2,
    LBKM_BC_DIRICHLET = 3,
    LBKM_BC_SPECULAR = 4,
    LBKM_BC_SIDES = 5
} lbkm_bc;

typedef struct {
    int32_t nx, ny;        /* grid; ny = 1 for one-dimensional runs */
    int32_t precision;     /* lbkm_precision */
    int32_t recovery;      /* lbkm_recovery, used by LBKM_F32 only */
    double gamma;          /* specific-heat ratio; I = 2/(gamma-1) - D (Sec. III) */
    double Pr;             /* if > 0: S_8 = S_9 = Pr * S_5 (Pr = R_kappa/R_mu,
                              Sec. III, needs S_5 = S_6 = S_7); if <= 0: S as given */
    int32_t orbit_kind[4]; /* must be {0, 1, 0, 1} (axis, diagonal, axis, diagonal) */
    double orbit_speed[4]; /* v of each orbit (> 0) */
    double orbit_eta[4];   /* eta of each orbit (>= 0) */
    double S[16];          /* relaxation rates R_1..R_16 (R_1..R_4 accepted, unused,
                              Sec. III); require dt * max(S_5..S_16) < 2 */
    double Q;              /* heat release per unit mass (Eq. (18)) */
    double omega1, omega2; /* Cochran rate constants of Eq. (28), m = n = 1 */
    double T_ig;           /* reaction only where T > T_ig (Sec. II); finite, >= 0 */
    double dx, dy, dt;     /* grid spacing and time step */
    int32_t bc_x, bc_y;    /* lbkm_bc for each direction */
    int32_t tne_every;     /* 0: no on-the-fly TNE; k > 0: reduce the TNE of the
                              input state of every k-th step into the history (the
                              FP32 2-D step then gathers the statistics on every step
                              and reduces them on the k-th: a step costs the same for
                              any k > 0, and with 0 it carries no TNE work at all) */
    int32_t tne_capacity;  /* records kept in the device history ring (>= 1) */
    double wall_ux[2], wall_uy[2], wall_T[2]; /* bc_y = LBKM_BC_WALL: velocity and
                              temperature of the wall below row 0 ([0]) and above
                              row ny-1 ([1]); T_w > 0 */
    int32_t side_bc[4];    /* with LBKM_BC_SIDES: conditions of the sides x = 0, x = nx,
                              y = 0, y = ny (see lbkm_bc) */
    double side_rho[4], side_ux[4], side_uy[4], side_T[4], side_lam[4]; /* Dirichlet
                              states of those sides; rho > 0, T > 0 */
    int32_t time_scheme;   /* 0: forward Euler (the paper's single stage); 1: two-stage
                              SSP Runge-Kutta from that step E, u^{n+1} = (u^n +
                              E(E(u^n)))/2 (second order in time; two launches per
                              step); 2: three-stage SSP Runge-Kutta (Shu-Osher form),
                              u2 = 3/4 u^n + 1/4 E(E(u^n)), u^{n+1} = 1/3 u^n + 2/3 E(u2)
                              (third order; three launches per step, a third state
                              copy); TNE of u^n; not for batched instances or lbkm_grad */
    int32_t collision;     /* 0: the single-relaxation-time fast path wherever it applies
                              (S_5..S_16 all equal, tne_every = 0, LBKM_F32 on a 2-D grid,
                              forward Euler, periodic or zero-gradient sides; Sec. V): the
                              collision -S (f - f^eq) + C of Eq. (87) in velocity space
                              needs one inverse transform and no forward one; 1: always
                              the moment-space form of Eq. (1) */
    /* Caller-owned device memory (an interface of this library, no counterpart in the
       paper): if alloc is not NULL, every device buffer of the handle and of its calls
       (states, TNE partials and history, counters, batched tables, temporaries of
       init_fields / macros / tne, workspaces of lbkm_grad and lbkm_autotune) comes from
       alloc(bytes, cuda_stream, alloc_ctx) and goes back through free(ptr, cuda_stream,
       alloc_ctx), with the handle's stream; a temporary is freed only after that stream
       has been synchronised. Blocks must be aligned to 256 bytes (else LBKM_EINVAL); NULL
       from alloc gives LBKM_ENOMEM. Set both or neither. */
    void* (*alloc)(size_t bytes, void* cuda_stream, void* ctx);
    void (*free)(void* ptr, void* cuda_stream, void* ctx);
    void* alloc_ctx;
} lbkm_params;

/* Grid-wide TNE measures of one state (Sec. VI). Sums are weighted by dx*dy;
 * min and max are unweighted. Index k-1 holds Delta_k; Delta_1..Delta_4 are 0. */
typedef struct {
    double sum[16], abs_sum[16], min[16], max[16];
    double d_sum, d2_sum; /* sum of d and of d^2, d = sqrt(sum_k Delta_k^2) */
    int64_t step;         /* step index of the state the record describes */
} lbkm_tne_global;

/* Fill *p with defaults: D2V16 orbits (axis 2.7/eta 5, diagonal 2.2/eta 0,
 * axis 1.2/eta 3, diagonal 1.0/eta 0), gamma 1.4, S_k = 1e5, Q = 0, T_ig = 1.1,
 * dx = dy = 1e-3, dt = 1e-5, zero-gradient x, periodic y, LBKM_F64, TNE off,
 * tne_capacity 1. nx, ny are set to 0 and must be filled in.
 * The default orbits carry the Sod tube, the steady detonation, the 2-D reactive field
 * and Couette flow. Stronger shocks need faster orbits: the Lax tube runs with these
 * speeds times 1.5, and the regular shock reflection of Sec. IV.C stays stable with them
 * only to t ~ 0.11 (then it breaks down behind the reflection point, in the oracle too);
 * the D2V24 handle (lbkm24.h) runs it to t = 0.5 with the paper's own set. */
void lbkm_default_params(lbkm_params* p);

/* Validate p, build M (rows m_1..m_16), invert it in block form and keep the
 * model constants for kernel-parameter (constant-bank) delivery, allocate the
 * two device copies of the state [17][ny][pitch] (f_1..f_16, lambda) and the
 * reduction buffers. cuda_stream: a cudaStream_t (NULL = legacy default stream)
 * on the current device; the handle launches all its work there.
 * Errors: LBKM_EINVAL (bad sizes or parameters, message names the field),
 * LBKM_ESINGULAR, LBKM_ENOMEM, LBKM_ECUDA. On error *out is NULL. */
lbkm_status lbkm_create(const lbkm_params* p, void* cuda_stream, lbkm_t* out);

/* Release every device and host resource of h (NULL is ignored). Synchronises
 * the handle's stream first. */
void lbkm_destroy(lbkm_t h);

/* Change the stream later work is launched on. */
lbkm_status lbkm_set_stream(lbkm_t h, void* cuda_stream);

/* Equilibrium start, f = M^-1 f_hat^eq(rho, u, T) (Eq. (16)), and lambda.
 * rho, ux, uy, T, lambda: [ny][nx] FP64, host (on_device = 0) or device. Host
 * fields that are all page-locked (pinned) are read by the kernel in place; others
 * go through a device temporary. lambda may be NULL (then lambda = 0). Resets the
 * step counter to 0 and the TNE history. Synchronises.
 * Errors: LBKM_EINVAL (NULL field), LBKM_ECUDA. */
lbkm_status lbkm_init_fields(lbkm_t h, const double* rho, const double* ux, const double* uy,
                             const double* T, const double* lambda, int on_device);

/* Advance n >= 0 time steps, asynchronously on the handle's stream. Each step
 * (each stage of a Runge-Kutta step) is one fused kernel (stencil, collision,
 * reaction, Euler update and, when due, the per-block TNE partials); on steps that
 * reduce TNE a small kernel then folds the partials into the history record.
 * Repeated chunks are replayed from a CUDA graph.
 * Errors: LBKM_ESTATE (no init_fields yet), LBKM_EINVAL (n < 0), LBKM_ECUDA. */
lbkm_status lbkm_step(lbkm_t h, int64_t n);

/* Wait for the handle's stream and check the device status word.
 * Errors: LBKM_EUNSTABLE, LBKM_ECUDA. */
lbkm_status lbkm_sync(lbkm_t h);

/* Number of steps taken since lbkm_init_fields / lbkm_set_state. */
int64_t lbkm_steps_taken(lbkm_t h);

/* Macroscopic fields of the current state (Eqs. (5)-(7)): rho, u_x, u_y, T,
 * p = rho T and lambda, each [ny][nx] FP64, host or device; NULL pointers are
 * skipped. Host outputs that are all page-locked (pinned) are written by the kernel in
 * place; others through a device temporary. Synchronises.
 * Errors: LBKM_ESTATE, LBKM_EUNSTABLE, LBKM_ECUDA. */
lbkm_status lbkm_macros(lbkm_t h, double* rho, double* ux, double* uy, double* T, double* p,
                        double* lambda, int on_device);

/* TNE of the current state (Sec. VI): delta, if not NULL, receives
 * Delta_1..Delta_16 as [16][ny][nx] FP64 (host or device, Delta_1..4 = 0);
 * g, if not NULL, receives the grid-wide record (host memory). Synchronises. */
lbkm_status lbkm_tne(lbkm_t h, double* delta, lbkm_tne_global* g, int on_device);

/* Copy up to max_records of the on-the-fly TNE records, oldest first, to out
 * (host). *n_out receives how many were copied. Records older than
 * tne_capacity steps are overwritten. Synchronises. */
lbkm_status lbkm_tne_history(lbkm_t h, lbkm_tne_global* out, int32_t max_records,
                             int32_t* n_out);

/* Bytes of one state snapshot (17 planes of nx*ny values in the handle's
 * precision, FP64 or FP32, row-major, f_1..f_16 then lambda, followed by the
 * int64 step counter). */
size_t lbkm_state_bytes(lbkm_t h);

/* Checkpoint / resume: copy the current state to dst or load it from src
 * (lbkm_state_bytes() bytes, host or device). set_state clears the status word
 * and the TNE history. Errors: LBKM_EINVAL, LBKM_ESTATE, LBKM_ECUDA. */
lbkm_status lbkm_get_state(lbkm_t h, void* dst, int on_device);
lbkm_status lbkm_set_state(lbkm_t h, const void* src, int on_device);

/* TNE record of a caller-owned state, allocating nothing (the paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory, e.g. because their own pool already holds all of it, or because a
 * latency-bound loop must not pay cudaMalloc's implicit synchronisation).
 * No handle is needed: p gives the model (nx, ny, precision, gamma, orbits,
 * dx, dy; the rest is ignored), state is a device array of 17 planes [ny][pitch]
 * in p->precision (f_1..f_16, lambda; the layout lbkm_get_state writes with
 * pitch = nx), delta is NULL or a device array [16][ny][nx] FP64, and out is a
 * device pointer to one lbkm_tne_global (step is set to -1). The call is
 * asynchronous on cuda_stream. Scratch: a fixed device array inside the library
 * (about 0.8 MB on every GPU that loads it, kept until the process exits),
 * shared by all calls: calls that overlap on the GPU race, so serialise them
 * (one stream, or events). Each call outside stream capture looks up the
 * scratch address with the calling device current (so a device reset or a new
 * primary context is followed); a call during capture uses the address the
 * last such lookup on that device found, so the first call on a device must
 * come before any stream capture (else LBKM_ESTATE). Limits: nx * ny <=
 * 16,777,216 cells and nx <= pitch <= 2,147,483,647 elements; other values
 * return LBKM_EINVAL. Errors: LBKM_EINVAL, LBKM_ESINGULAR, LBKM_ESTATE,
 * LBKM_ECUDA, with the message in lbkm_last_error(NULL). */
lbkm_status lbkm_tne_noalloc(const lbkm_params* p, const void* state, int64_t pitch,
                             double* delta, lbkm_tne_global* out, void* cuda_stream);

/* Objective of lbkm_grad over N steps from the handle's current state (t = 0):
 * J = w_mismatch/2 sum_x (rho_N - rho*)^2 dx + w_tne sum_{n<N} sum_x d_n^2 dx dt,
 * d_n^2 = sum_k Delta_k^2 of the state entering step n (Sec. VI, Eqs. (90)-(91)). */
typedef struct {
    const double* rho_target;  /* [nx] host: rho* */
    double w_mismatch, w_tne;
    int64_t steps;             /* N >= 1 */
    int32_t checkpoint_every;  /* a state is kept every this many steps (>= 1) */
} lbkm_objective;

typedef struct {
    double J, J_mismatch, J_tne;
    double dS[16];             /* dJ/dS_1..16 (S_1..4: 0, Sec. III) */
    double dQ, domega1;        /* dJ/dQ, dJ/domega1 */
    double* drho0;             /* [nx] host or NULL: dJ/drho of the start, with u, T fixed,
                                  for a start made by lbkm_init_fields (equilibrium) */
    double* df0;               /* [16][nx] host or NULL: dJ/df of the start state */
    double domega2;            /* dJ/domega2 (Eq. (28); defined at omega2 = 0 too) */
} lbkm_grad_out;

/* Gradient of J by the discrete adjoint of the step (reverse mode through every
 * step, hand-written FP64 kernels): the forward run keeps a state every
 * checkpoint_every steps and each segment is recomputed from its checkpoint
 * before its steps are reversed, so memory is (N/C + C) states. With an LBKM_F32
 * handle the forward run is the FP32 step and its checkpoints are FP32 states; each
 * segment is then recomputed in FP64 from its checkpoint widened to FP64 and reversed
 * in FP64 (J and its derivative are those of FP64 segments restarted from the FP32
 * run's states). The exact adjoint of the FP32 step itself is not offered: over long
 * runs FP32 rounding decides the limiter's branches on flat stretches every step, and
 * the limiter's linearisation about such states amplifies the adjoint. The reaction's
 * derivative covers omega2 != 0 (the closed form of Eq. (28)). The ignition
 * switch T > T_ig stays a hard switch (no derivative through it); minmod and the
 * lambda clamp follow the branch the forward values take. The handle's state is
 * left unchanged. Needs a handle with ny = 1, periodic (nx >= 5) or zero-gradient ends and
 * forward Euler (not batched). Errors: LBKM_EINVAL, LBKM_ESTATE, LBKM_ENOMEM,
 * LBKM_ECUDA, LBKM_EUNSTABLE. Synchronises. */
lbkm_status lbkm_grad(lbkm_t h, const lbkm_objective* obj, lbkm_grad_out* out);

/* The objective J of lbkm_grad alone (same definition, Sec. VI, Eqs. (90)-(91); for an
 * LBKM_F32 handle the same FP64 segments restarted every checkpoint_every steps from the
 * FP32 run's states), without its derivative: the run and one d^2 reduction per state,
 * no reverse sweep and no checkpoints kept. *J receives J; J_mismatch and J_tne (each
 * may be NULL) its two terms. It agrees with lbkm_grad's J up to the order of the FP64
 * additions. Same conditions and errors as lbkm_grad; the handle's state is left
 * unchanged. Synchronises. */
lbkm_status lbkm_objective_value(lbkm_t h, const lbkm_objective* obj, double* J,
                                 double* J_mismatch, double* J_tne);

/* Many independent 1-D instances of uneven length in one handle (zero-gradient
 * boundaries per instance), advanced together by one persistent kernel per
 * chunk of steps (replayed from a CUDA graph). p gives everything the instances
 * share (velocity set, gamma, Pr, omega2, T_ig, dx, dt; precision must be
 * LBKM_F32, tne_every 0); p->nx, p->ny, p->bc_x are ignored. inst_nx[i]: cells
 * of instance i (a multiple of 4, >= 4). inst_S ([n][16]), inst_Q ([n]),
 * inst_omega1 ([n]): per-instance rates, heat release and rate constant, or
 * NULL to use p->S, p->Q, p->omega1 for all. The fields of lbkm_init_fields,
 * lbkm_macros, lbkm_tne and the state of lbkm_get_state are the instances
 * concatenated in order (nx = sum inst_nx, ny = 1). Errors as lbkm_create. */
lbkm_status lbkm_create_batched(const lbkm_params* p, int32_t n_instances,
                                const int32_t* inst_nx, const double* inst_S,
                                const double* inst_Q, const double* inst_omega1,
                                void* cuda_stream, lbkm_t* out);

/* Number of instances of h (1 for a single grid). */
int32_t lbkm_instances(lbkm_t h);

/* TNE record (Sec. VI) of each instance of a batched handle, FP64, into out
 * (host, lbkm_instances(h) records, step = -1). Synchronises. */
lbkm_status lbkm_tne_instances(lbkm_t h, lbkm_tne_global* out);

/* Choose the block size and the number of resident blocks of the persistent
 * kernel by timing trial_steps steps of each candidate on the handle's own
 * state, which is restored afterwards. chosen (3 ints, may be NULL) receives
 * threads per block, blocks per SM and blocks. Synchronises. Single grids keep
 * their fixed plan (chosen = 0). */
lbkm_status lbkm_autotune(lbkm_t h, int32_t trial_steps, int32_t* chosen);

/* Bound of each grid-barrier wait of the persistent kernel (default 2 s). A
 * wait that runs out sets the status word; the next synchronising call returns
 * LBKM_ETIMEOUT and the kernel has returned instead of hanging.
 * phantom_blocks > 0 makes the barrier wait for blocks that do not exist: for
 * testing that path only. */
lbkm_status lbkm_set_wait_limit(lbkm_t h, int64_t timeout_ns, int32_t phantom_blocks);

/* Message of the last failing call on h (or of the last failing lbkm_create
 * when h is NULL). Never NULL. */
const char* lbkm_last_error(lbkm_t h);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t lbkm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBKM_H */
