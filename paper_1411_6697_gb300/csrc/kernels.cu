// kernels.cu -- CUDA kernels of the MRT-LBKM step for sm_103a.
//
// step_kernel: one fused forward-Euler stage of the FP64 form and of FP32 1-D grids
// (FP32 2-D grids run march_kernel, march.cu). Each block walks tiles of
// TX x TY cells (grid-stride loop, grid = SMs x resident blocks). Per tile it
//   1. stages the 17 planes (f_1..f_16, lambda) of the tile plus a 2-cell halo
//      in shared memory (coalesced row loads, boundary condition applied by
//      index mapping);
//   2. recovers rho, u, T of the tile and a 1-cell ring (needed by grad u) from
//      the conserved moments, in FP64 or double-float;
//   3. per cell: moments by butterflies + sector blocks, f_hat^eq, Delta_k,
//      A_hat_8/9 (Eqs. (3)-(4)), reaction (Eq. (28)), C_hat (Eqs. (19)-(23)),
//      Omega = M^-1 Omega_hat, NND flux differences of v_i f_i from shared
//      memory, Euler update, lambda update; each f_i is read once from HBM and
//      written once;
//   4. when the TNE of this step is due, accumulates Delta_k statistics
//      (warp shuffles, then FP64 per warp), and the last block to finish
//      reduces the per-block partials in a fixed order (deterministic).
// The plain FP64 form instantiates the same kernel with R = double.
#include <float.h>

#include "cell.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace lbk {

namespace {

template <typename R, bool TWO_D, int TX, int TY>
struct Cfg {
    static constexpr int H = TWO_D ? 2 : 0;  // halo rows of f (NND radius)
    static constexpr int H1 = TWO_D ? 1 : 0; // ring rows of macros (grad u)
    static constexpr int SW = TX + 4, SH = TY + 2 * H, PS = SW * SH;
    static constexpr int RW = TX + 2, RH = TY + 2 * H1, RS = RW * RH;
    static constexpr int NT = TX * TY, NW = NT / 32;
    static constexpr size_t off_mac = ((size_t)NPLANE * PS * sizeof(R) + 15) / 16 * 16;
    static constexpr size_t off_Td = off_mac + 4 * RS * sizeof(R);
    static constexpr size_t off_off = (off_Td + RS * sizeof(double) + 15) / 16 * 16;
    static constexpr size_t off_tsum = off_off;
    static constexpr size_t off_tmm = off_tsum + (size_t)NW * NSUM * sizeof(double);
    static constexpr size_t smem = off_tmm + (size_t)NW * NMM * sizeof(R);
};

template <typename R, int REC, bool TWO_D, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
    step_kernel(const ModelConst<R> K, const StepLaunch a)
{
    using C = Cfg<R, TWO_D, TX, TY>;
    extern __shared__ __align__(16) unsigned char smem[];
    R* sf = reinterpret_cast<R*>(smem);
    R* smac = reinterpret_cast<R*>(smem + C::off_mac); // rho, ux, uy, T  [4][RH][RW]
    double* sTd = reinterpret_cast<double*>(smem + C::off_Td);
    double* tsum = reinterpret_cast<double*>(smem + C::off_tsum);
    R* tmm = reinterpret_cast<R*>(smem + C::off_tmm);

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int warp = tid >> 5, lane = tid & 31;
    const int nx = K.nx, ny = K.ny, pitch = K.pitch;
    const int64_t plane = K.plane;
    const R* __restrict__ in = static_cast<const R*>(a.in);
    R* out = static_cast<R*>(a.out); // not restrict: prev may alias it

    const int64_t step = a.ctr->step;
    const bool do_tne = a.tne_every > 0 && (step % a.tne_every) == 0 && a.stage < 2;
    const bool avg = a.stage >= 2; // later SSP-RK stage: weighted with u^n (prev)
    const R* prev = static_cast<const R*>(a.prev);
    const R wp = (R)a.wprev, wn = (R)a.wnew;
    if (do_tne) {
        for (int i = tid; i < C::NW * NSUM; i += C::NT) tsum[i] = 0.0;
        for (int i = tid; i < C::NW * NMM; i += C::NT)
            tmm[i] = (i % NMM) < TNE_K ? big_value<R>() : -big_value<R>();
    }
    int bad = 0;

    const int tiles_x = (nx + TX - 1) / TX;
    const int tiles_y = (ny + TY - 1) / TY;
    const int ntiles = tiles_x * tiles_y;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        __syncthreads();
        // 1. stage f and lambda with halo
        for (int idx = tid; idx < NPLANE * C::PS; idx += C::NT) {
            const int p = idx / C::PS;
            const int rem = idx - p * C::PS;
            const int r = rem / C::SW, c = rem - r * C::SW;
            sf[idx] = ghost_value(K, in, p, x0 - 2 + c, TWO_D ? y0 - C::H + r : y0);
        }
        __syncthreads();
        if constexpr (TWO_D) {
            // walls: the staged ghost rows hold copies of the edge fluid row (the
            // index map clamps); add the non-equilibrium-extrapolation correction
            if ((K.sbc[2] == 2 || K.sbc[3] == 2) && (y0 - C::H < 0 || y0 + TY + C::H > ny)) {
                for (int idx = tid; idx < 2 * C::SW; idx += C::NT) {
                    const int side = idx / C::SW, c = idx - side * C::SW;
                    if (K.sbc[2 + side] != 2) continue;
                    const int rs = (side == 0 ? 0 : ny - 1) - (y0 - C::H); // fluid row
                    if (rs < 0 || rs >= C::SH) continue;
                    R fl[16], d[16];
#pragma unroll
                    for (int i = 0; i < 16; i++) fl[i] = sf[i * C::PS + rs * C::SW + c];
                    wall_correction(K, fl, side, d);
                    for (int r = 0; r < C::SH; r++) {
                        const int gy = y0 - C::H + r;
                        if (side == 0 ? gy >= 0 : gy < ny) continue;
#pragma unroll
                        for (int i = 0; i < 16; i++) sf[i * C::PS + r * C::SW + c] += d[i];
                    }
                }
                __syncthreads();
            }
        }
        // 2. macros of the tile and its ring
        for (int idx = tid; idx < C::RS; idx += C::NT) {
            const int r = idx / C::RW, c = idx - r * C::RW;
            const int s = (r + C::H - C::H1) * C::SW + c + 1;
            R fl[16];
#pragma unroll
            for (int i = 0; i < 16; i++) fl[i] = sf[i * C::PS + s];
            double rho, ux, uy, T;
            if constexpr (REC == 1)
                recover_df32(K.cd, K.wd, K.inv_DId, reinterpret_cast<const float*>(fl), rho, ux,
                             uy, T);
            else
                recover_f64(K.cd, K.wd, K.inv_DId, fl, rho, ux, uy, T);
            smac[idx] = (R)rho;
            smac[C::RS + idx] = (R)ux;
            smac[2 * C::RS + idx] = (R)uy;
            smac[3 * C::RS + idx] = (R)T;
            sTd[idx] = T;
        }
        __syncthreads();

        // 3. the cell update
        const int gx = x0 + lx, gy = y0 + ly;
        const bool active = gx < nx && gy < ny;
        R Dk[TNE_K];
        if (active) {
            const int c0 = (ly + C::H) * C::SW + lx + 2;
            const int m0 = (ly + C::H1) * C::RW + lx + 1;
            R f[16];
#pragma unroll
            for (int i = 0; i < 16; i++) f[i] = sf[i * C::PS + c0];
            const R lam0 = sf[16 * C::PS + c0];
            const R rho = smac[m0], ux = smac[C::RS + m0], uy = smac[2 * C::RS + m0];
            const R T = smac[3 * C::RS + m0];
            const double Td = sTd[m0];
            if (!(rho > R(0)) || !(Td > 0.0) || !isfinite(ux + uy + Td + (double)rho)) bad = 1;

            R m[16], q[16];
            forward_moments(K, f, m);
            feq_moments(K.DI, rho, ux, uy, T, q);
#pragma unroll
            for (int k = 0; k < TNE_K; k++) Dk[k] = m[k + 4] - q[k + 4];

            const R* sux = smac + C::RS;
            const R* suy = smac + 2 * C::RS;
            const R dux_dx = (sux[m0 + 1] - sux[m0 - 1]) * K.half_inv_dx;
            const R duy_dx = (suy[m0 + 1] - suy[m0 - 1]) * K.half_inv_dx;
            R dux_dy = R(0), duy_dy = R(0);
            if constexpr (TWO_D) {
                dux_dy = (sux[m0 + C::RW] - sux[m0 - C::RW]) * K.half_inv_dy;
                duy_dy = (suy[m0 + C::RW] - suy[m0 - C::RW]) * K.half_inv_dy;
            }
            const R theta = (dux_dx + duy_dy) * K.inv_DI;
            const R shear = duy_dx + dux_dy;
            const R rT = rho * T;
            const R A8 = rT * K.A8c * (R(4) * ux * (dux_dx - theta) + R(2) * uy * shear);
            const R A9 = rT * K.A9c * (R(4) * uy * (duy_dy - theta) + R(2) * ux * shear);

            R dlam = R(0);
            if (Td > K.T_igd) dlam = reaction_increment(lam0, K.omega1 * rT, K.omega2 * rT, K.dt);
            const R cr = dlam * K.chem;

            R dq[16], Om[16], W[16];
            dfeq_dT(K.DI, rho, ux, uy, T, dq);
            Om[0] = Om[1] = Om[2] = R(0);
            Om[3] = dq[3] * cr;
#pragma unroll
            for (int k = 4; k < 16; k++) Om[k] = fma(-K.S[k], Dk[k - 4], dq[k] * cr);
            Om[7] += A8;
            Om[8] += A9;
            inverse_moments(K, Om, W);

            // NND flux differences (compile-time upwind side per velocity)
            const R* s0 = sf + c0;
#define FV(i, ox, oy) s0[(i) * C::PS + (oy) * C::SW + (ox)]
#define PX(i) nnd_pos(FV(i, -2, 0), FV(i, -1, 0), FV(i, 0, 0), FV(i, 1, 0))
#define NX(i) nnd_neg(FV(i, -1, 0), FV(i, 0, 0), FV(i, 1, 0), FV(i, 2, 0))
#define PY(i) nnd_pos(FV(i, 0, -2), FV(i, 0, -1), FV(i, 0, 0), FV(i, 0, 1))
#define NY(i) nnd_neg(FV(i, 0, -1), FV(i, 0, 0), FV(i, 0, 1), FV(i, 0, 2))
            R adv[16];
#pragma unroll
            for (int o = 0; o < 2; o++) { // axis orbits 0, 2
                const int i0 = 8 * o;
                const R cx = K.c[2 * o] * K.inv_dx, cy = K.c[2 * o] * K.inv_dy;
                adv[i0 + 0] = cx * PX(i0 + 0);
                adv[i0 + 2] = -cx * NX(i0 + 2);
                if constexpr (TWO_D) {
                    adv[i0 + 1] = cy * PY(i0 + 1);
                    adv[i0 + 3] = -cy * NY(i0 + 3);
                } else {
                    adv[i0 + 1] = adv[i0 + 3] = R(0);
                }
            }
#pragma unroll
            for (int o = 0; o < 2; o++) { // diagonal orbits 1, 3
                const int i0 = 4 + 8 * o;
                const R cx = K.c[2 * o + 1] * K.inv_dx, cy = K.c[2 * o + 1] * K.inv_dy;
                R x0p = cx * PX(i0 + 0), x1n = cx * NX(i0 + 1), x2n = cx * NX(i0 + 2),
                  x3p = cx * PX(i0 + 3);
                R y0p = R(0), y1p = R(0), y2n = R(0), y3n = R(0);
                if constexpr (TWO_D) {
                    y0p = cy * PY(i0 + 0);
                    y1p = cy * PY(i0 + 1);
                    y2n = cy * NY(i0 + 2);
                    y3n = cy * NY(i0 + 3);
                }
                adv[i0 + 0] = x0p + y0p;
                adv[i0 + 1] = y1p - x1n;
                adv[i0 + 2] = -(x2n + y2n);
                adv[i0 + 3] = x3p - y3n;
            }
            const int64_t g = (int64_t)gy * pitch + gx;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const R v = f[i] + K.dt * (W[i] - adv[i]);
                out[i * plane + g] = avg ? wp * prev[i * plane + g] + wn * v : v;
            }

            // lambda: u . grad(lambda) with NND interface values, reaction, clamp
            R la = ux > R(0) ? ux * PX(16) : (ux < R(0) ? ux * NX(16) : R(0));
            la *= K.inv_dx;
            if constexpr (TWO_D) {
                R lb = uy > R(0) ? uy * PY(16) : (uy < R(0) ? uy * NY(16) : R(0));
                la += lb * K.inv_dy;
            }
#undef FV
#undef PX
#undef NX
#undef PY
#undef NY
            R ln = lam0 - K.dt * la + dlam;
            ln = ln < R(0) ? R(0) : (ln > R(1) ? R(1) : ln);
            out[16 * plane + g] = avg ? wp * prev[16 * plane + g] + wn * ln : ln;
        }

        // 4. TNE statistics of this tile (all lanes take part in the shuffles)
        if (do_tne) {
            R d2 = R(0);
#pragma unroll
            for (int k = 0; k < TNE_K; k++) {
                if (!active) Dk[k] = R(0);
                d2 += Dk[k] * Dk[k];
            }
#pragma unroll
            for (int k = 0; k < TNE_K; k++) {
                R s = warp_sum(Dk[k]);
                R sa = warp_sum(Dk[k] < R(0) ? -Dk[k] : Dk[k]);
                R mn = warp_min(active ? Dk[k] : big_value<R>());
                R mx = warp_max(active ? Dk[k] : -big_value<R>());
                if (lane == 0) {
                    tsum[warp * NSUM + k] += (double)s;
                    tsum[warp * NSUM + TNE_K + k] += (double)sa;
                    tmm[warp * NMM + k] = rmin(tmm[warp * NMM + k], mn);
                    tmm[warp * NMM + TNE_K + k] = rmax(tmm[warp * NMM + TNE_K + k], mx);
                }
            }
            R sd = warp_sum(sqrt(d2)), sd2 = warp_sum(d2);
            if (lane == 0) {
                tsum[warp * NSUM + 2 * TNE_K] += (double)sd;
                tsum[warp * NSUM + 2 * TNE_K + 1] += (double)sd2;
            }
        }
    }

    // end of step: status, TNE partials, arrival count; the last block finishes
    if (__syncthreads_or(bad) && tid == 0) atomicOr(&a.ctr->status, 1);
    if (do_tne) {
        double* part = a.partials + blockIdx.x; // quantity-major, stride gridDim.x
        const size_t ps = gridDim.x;
        for (int q = tid; q < NSUM; q += C::NT) {
            double s = 0.0;
            for (int w = 0; w < C::NW; w++) s += tsum[w * NSUM + q];
            part[ps * (q < 2 * TNE_K ? q : 4 * TNE_K + (q - 2 * TNE_K))] = s;
        }
        for (int q = tid; q < NMM; q += C::NT) {
            R v = tmm[q];
            for (int w = 1; w < C::NW; w++)
                v = q < TNE_K ? rmin(v, tmm[w * NMM + q]) : rmax(v, tmm[w * NMM + q]);
            part[ps * (2 * TNE_K + q)] = (double)v;
        }
        __threadfence();
    }
    __syncthreads();
    __shared__ unsigned int s_last;
    if (tid == 0) s_last = (atomicAdd(&a.ctr->arrivals, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last && tid == 0) { // the grid-wide TNE record is finished by launch_tne_finish
        if (do_tne) {
            a.ctr->hist_count += 1;
            a.ctr->tne_step = step;
        }
        if (a.stage < 2) a.ctr->tne_pending = do_tne ? 1 : 0;
        if (a.stage == 0 || a.stage == 2) a.ctr->step = step + 1;
        a.ctr->arrivals = 0u;
    }
}

template <typename R, int REC, bool TWO_D, int TX, int TY>
struct StepKernel {
    using C = Cfg<R, TWO_D, TX, TY>;
    // opt in to the dynamic shared memory once per process, before any capture
    static cudaError_t prepare()
    {
        static cudaError_t done = cudaFuncSetAttribute(
            step_kernel<R, REC, TWO_D, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)C::smem);
        return done;
    }
    static int grid(int nx, int ny)
    {
        static int per_sm = -1, sms = -1;
        if (per_sm < 0) {
            if (prepare() != cudaSuccess) return -1;
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, step_kernel<R, REC, TWO_D, TX, TY>, C::NT, C::smem) != cudaSuccess)
                return -1;
            if (per_sm < 1) per_sm = 1;
        }
        long tiles = (long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
        long g = (long)per_sm * sms;
        return (int)(tiles < g ? tiles : g);
    }
    static cudaError_t launch(const void* K, const StepLaunch& a, cudaStream_t s)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        step_kernel<R, REC, TWO_D, TX, TY><<<a.grid, C::NT, C::smem, s>>>(
            *static_cast<const ModelConst<R>*>(K), a);
        return cudaGetLastError();
    }
};

// tile shapes: 2-D 32 x 8 cells, 1-D 64 cells
template <typename R, int REC>
using K2D = StepKernel<R, REC, true, 32, 8>;
template <typename R, int REC>
using K1D = StepKernel<R, REC, false, 64, 1>;

// ------------------------------------------------------------ init, macros, TNE
template <typename R>
__global__ void init_kernel(const ModelConst<double> K, const double* rho, const double* ux,
                            const double* uy, const double* T, const double* lam, R* state)
{
    const int64_t n = (int64_t)K.nx * K.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / K.nx), x = (int)(c - (int64_t)y * K.nx);
        double q[16], f[16];
        feq_moments(K.DI, rho[c], ux[c], uy[c], T[c], q);
        inverse_moments(K, q, f);
        const int64_t g = (int64_t)y * K.pitch + x;
#pragma unroll
        for (int i = 0; i < 16; i++) state[i * K.plane + g] = (R)f[i];
        state[16 * K.plane + g] = (R)(lam ? lam[c] : 0.0);
    }
}

template <typename R>
__global__ void macros_kernel(const ModelConst<double> K, const R* state, double* rho,
                              double* ux, double* uy, double* T, double* p, double* lam)
{
    const int64_t n = (int64_t)K.nx * K.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / K.nx), x = (int)(c - (int64_t)y * K.nx);
        const int64_t g = (int64_t)y * K.pitch + x;
        R f[16];
#pragma unroll
        for (int i = 0; i < 16; i++) f[i] = state[i * K.plane + g];
        double r, u, v, t;
        recover_f64(K.cd, K.wd, K.inv_DId, f, r, u, v, t);
        if (rho) rho[c] = r;
        if (ux) ux[c] = u;
        if (uy) uy[c] = v;
        if (T) T[c] = t;
        if (p) p[c] = r * t;
        if (lam) lam[c] = (double)state[16 * K.plane + g];
    }
}

constexpr int TNE_THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(TNE_THREADS)
    tne_kernel(const ModelConst<double> K, const R* state, double* delta, double* partials,
               DevCounters* ctr, TneRecord* out, double area)
{
    __shared__ double ssum[TNE_THREADS / 32][NSUM];
    __shared__ double smm[TNE_THREADS / 32][NMM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[NSUM], mn[TNE_K], mx[TNE_K];
    for (int q = 0; q < NSUM; q++) acc[q] = 0.0;
    for (int k = 0; k < TNE_K; k++) mn[k] = DBL_MAX, mx[k] = -DBL_MAX;
    const int64_t n = (int64_t)K.nx * K.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / K.nx), x = (int)(c - (int64_t)y * K.nx);
        const int64_t g = (int64_t)y * K.pitch + x;
        double f[16], m[16], q[16];
#pragma unroll
        for (int i = 0; i < 16; i++) f[i] = (double)state[i * K.plane + g];
        forward_moments(K, f, m);
        const double r = m[0], u = m[1] / r, v = m[2] / r;
        const double t = (m[3] / r - (u * u + v * v)) * K.inv_DId;
        feq_moments(K.DI, r, u, v, t, q);
        double d2 = 0.0;
        for (int k = 0; k < 16; k++) {
            double D = k < 4 ? 0.0 : m[k] - q[k];
            if (delta) delta[k * n + c] = D;
            if (k >= 4) {
                acc[k - 4] += D;
                acc[TNE_K + k - 4] += fabs(D);
                mn[k - 4] = fmin(mn[k - 4], D);
                mx[k - 4] = fmax(mx[k - 4], D);
                d2 += D * D;
            }
        }
        acc[2 * TNE_K] += sqrt(d2);
        acc[2 * TNE_K + 1] += d2;
    }
    for (int q = 0; q < NSUM; q++) {
        double s = warp_sum(acc[q]);
        if (lane == 0) ssum[warp][q] = s;
    }
    for (int k = 0; k < TNE_K; k++) {
        double a = warp_min(mn[k]), b = warp_max(mx[k]);
        if (lane == 0) smm[warp][k] = a, smm[warp][TNE_K + k] = b;
    }
    __syncthreads();
    double* part = partials + blockIdx.x; // quantity-major, stride gridDim.x
    const size_t ps = gridDim.x;
    if (threadIdx.x < NSUM) {
        double s = 0.0;
        for (int w = 0; w < TNE_THREADS / 32; w++) s += ssum[w][threadIdx.x];
        const int q = threadIdx.x;
        part[ps * (q < 2 * TNE_K ? q : 4 * TNE_K + (q - 2 * TNE_K))] = s;
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + NMM) {
        const int q = threadIdx.x - 32;
        double v = smm[0][q];
        for (int w = 1; w < TNE_THREADS / 32; w++)
            v = q < TNE_K ? fmin(v, smm[w][q]) : fmax(v, smm[w][q]);
        part[ps * (2 * TNE_K + q)] = v;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int s_last;
    if (threadIdx.x == 0) s_last = (atomicAdd(&ctr->arrivals, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (s_last) {
        __threadfence();
        finish_tne(partials, gridDim.x, out, ctr->step, area);
        __syncthreads();
        if (threadIdx.x == 0) ctr->arrivals = 0u;
    }
}

int sm_count()
{
    static int sms = -1;
    if (sms < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

int elementwise_grid(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * 16;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

} // namespace

static bool general_sides(const int sbc[4])
{
    return sbc[0] >= 2 || sbc[1] >= 2 || sbc[2] >= 2 || sbc[3] >= 2;
}

namespace {
constexpr int FIN_THREADS = 256;

// Block q reduces quantity q of the step's partials (quantity-major: partials[q *
// nblocks + b]) in a fixed order -- thread t takes blocks t, t + 256, ..., then the
// lanes in a shuffle tree and the warps in order -- and writes it into the record.
__global__ void __launch_bounds__(FIN_THREADS)
    tne_finish_kernel(const double* __restrict__ partials, int nblocks, TneRecord* hist,
                      int hist_cap, const DevCounters* ctr, double area)
{
    if (!ctr->tne_pending) return;
    __shared__ double wsum[FIN_THREADS / 32];
    const int q = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int kind = tne_kind(q);
    double acc = kind == 0 ? 0.0 : (kind == 1 ? DBL_MAX : -DBL_MAX);
    const double* pq = partials + (size_t)q * nblocks;
    for (int b = t; b < nblocks; b += FIN_THREADS) acc = tne_comb(kind, acc, __ldcg(pq + b));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = tne_comb(kind, acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) wsum[w] = acc;
    __syncthreads();
    if (t != 0) return;
    for (int k = 1; k < FIN_THREADS / 32; k++) acc = tne_comb(kind, acc, wsum[k]);
    TneRecord* rec = hist + (ctr->hist_count - 1) % hist_cap;
    if (q < TNE_K) rec->sum[q + 4] = acc * area;
    else if (q < 2 * TNE_K) rec->abs_sum[q - TNE_K + 4] = acc * area;
    else if (q < 3 * TNE_K) rec->min[q - 2 * TNE_K + 4] = acc;
    else if (q < 4 * TNE_K) rec->max[q - 3 * TNE_K + 4] = acc;
    else if (q == 4 * TNE_K) rec->d_sum = acc * area;
    else rec->d2_sum = acc * area;
    if (q == 0) {
        for (int k = 0; k < 4; k++) rec->sum[k] = rec->abs_sum[k] = rec->min[k] = rec->max[k] = 0.0;
        rec->step = ctr->tne_step;
    }
}
} // namespace

cudaError_t launch_tne_finish(const StepLaunch& a, cudaStream_t s)
{
    tne_finish_kernel<<<TNE_PART, FIN_THREADS, 0, s>>>(a.partials, a.grid, a.hist, a.hist_cap,
                                                       a.ctr, a.cell_area);
    return cudaGetLastError();
}

int step_grid(int precision, int recovery, bool two_d, int nx, int ny, const int sbc[4])
{
    if (precision == 0)
        return two_d ? K2D<double, 0>::grid(nx, ny) : K1D<double, 0>::grid(nx, ny);
    if (two_d) return march_grid(recovery | (general_sides(sbc) ? 2 : 0), nx, ny);
    return recovery == 1 ? K1D<float, 1>::grid(nx, ny) : K1D<float, 0>::grid(nx, ny);
}

cudaError_t launch_step(int precision, int recovery, bool two_d, const void* K,
                        const StepLaunch& a, cudaStream_t s)
{
    if (precision == 0)
        return two_d ? K2D<double, 0>::launch(K, a, s) : K1D<double, 0>::launch(K, a, s);
    if (two_d) {
        const ModelConst<float>& Kf = *static_cast<const ModelConst<float>*>(K);
        return launch_march(recovery | (general_sides(Kf.sbc) ? 2 : 0) | (a.srt ? 4 : 0), Kf, a, s);
    }
    return recovery == 1 ? K1D<float, 1>::launch(K, a, s) : K1D<float, 0>::launch(K, a, s);
}

cudaError_t launch_init(int precision, const ModelConst<double>& Kd, const double* rho,
                        const double* ux, const double* uy, const double* T, const double* lam,
                        void* state, cudaStream_t s)
{
    const int64_t n = (int64_t)Kd.nx * Kd.ny;
    const int g = elementwise_grid(n, 256);
    if (precision == 0)
        init_kernel<double><<<g, 256, 0, s>>>(Kd, rho, ux, uy, T, lam, (double*)state);
    else
        init_kernel<float><<<g, 256, 0, s>>>(Kd, rho, ux, uy, T, lam, (float*)state);
    return cudaGetLastError();
}

cudaError_t launch_macros(int precision, const ModelConst<double>& Kd, const void* state,
                          double* rho, double* ux, double* uy, double* T, double* p,
                          double* lam, cudaStream_t s)
{
    const int64_t n = (int64_t)Kd.nx * Kd.ny;
    const int g = elementwise_grid(n, 256);
    if (precision == 0)
        macros_kernel<double><<<g, 256, 0, s>>>(Kd, (const double*)state, rho, ux, uy, T, p, lam);
    else
        macros_kernel<float><<<g, 256, 0, s>>>(Kd, (const float*)state, rho, ux, uy, T, p, lam);
    return cudaGetLastError();
}

int tne_grid(int nx, int ny) { return elementwise_grid((int64_t)nx * ny, TNE_THREADS); }

cudaError_t launch_tne(int precision, const ModelConst<double>& Kd, const void* state,
                       double* delta, double* partials, int grid, DevCounters* ctr,
                       TneRecord* out, double area, cudaStream_t s)
{
    if (precision == 0)
        tne_kernel<double><<<grid, TNE_THREADS, 0, s>>>(Kd, (const double*)state, delta,
                                                        partials, ctr, out, area);
    else
        tne_kernel<float><<<grid, TNE_THREADS, 0, s>>>(Kd, (const float*)state, delta, partials,
                                                       ctr, out, area);
    return cudaGetLastError();
}

} // namespace lbk
