// batch.cu -- persistent driver for many 1-D instances of uneven length.
//
// The instances are concatenated into one flat grid (each starts on a 16-byte
// boundary: nx is a multiple of 4). Work items are (instance, segment of 2*BT
// cells). One launch runs `nsteps` time steps: in each step the blocks walk the
// item list (grid-stride), staging segment + halo of the 17 planes with
// double-buffered cp.async copies, recovering rho, u, T of the segment and its
// two neighbours, and updating two cells per thread with packed FP32 pairs;
// boundaries are zero-gradient per instance, S, Q and omega1 per instance. A
// grid barrier separates the steps; its wait is bounded in time and reports a
// timeout through the status word instead of hanging. The launch is
// cooperative, so all blocks are resident.
#include <float.h>
#include <stdint.h>

#include "cell.cuh"
#include "kernels.cuh"
#include "pair.cuh"
#include "vec2.cuh"

namespace lbk {

namespace {

template <int BT>
struct BCfg {
    static constexpr int SEG = 2 * BT;           // cells per item
    static constexpr int SW = SEG + 8;           // staged: x0-4 .. x0+SEG+3
    static constexpr int CH = SW / 4;            // 16-byte chunks per plane
    static constexpr int MWB = SEG + 4;          // macro row: x0-2 .. x0+SEG+1
    static constexpr size_t OFF_MAC = (size_t)2 * NPLANE * SW * 4;
    static constexpr size_t OFF_IGN = OFF_MAC + (size_t)4 * MWB * 4;
    static constexpr size_t OFF_PAR = (OFF_IGN + SEG + 15) / 16 * 16;
    static constexpr size_t SMEM = OFF_PAR + 32 * 4;
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All blocks arrive; the last one advances the generation. A waiting block gives
// up after b.wait_ns nanoseconds, sets status bit 1 and reports false.
__device__ bool grid_barrier(const BatchLaunch& b, unsigned expected)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = b.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(b.bar, 1u) + 1u;
        if (arrived == expected) {
            b.bar[0] = 0u;
            __threadfence();
            atomicAdd(b.bar + 1, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > (uint64_t)b.wait_ns) {
                    atomicOr(&b.ctr->status, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <int BT>
__device__ __forceinline__ void stage_item(const float* __restrict__ in, float* buf,
                                           const InstParam& ip, int x0, int64_t plane)
{
    using C = BCfg<BT>;
    for (int c = threadIdx.x; c < NPLANE * C::CH; c += BT) {
        const int p = c / C::CH, ch = c - p * C::CH;
        const int x = x0 - 4 + 4 * ch;
        float* dst = buf + p * C::SW + 4 * ch;
        const float* src = in + p * plane + ip.off;
        if (x >= 0 && x + 4 <= ip.nx) {
            cp16(dst, src + x);
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                int xe = x + e;
                xe = xe < 0 ? 0 : (xe >= ip.nx ? ip.nx - 1 : xe);
                dst[e] = src[xe];
            }
        }
    }
}

template <int REC, int BT>
__global__ void __launch_bounds__(BT)
    batch_kernel(const ModelConst<float> K, const BatchLaunch b)
{
    using C = BCfg<BT>;
    extern __shared__ __align__(16) unsigned char smem[];
    float* stage = reinterpret_cast<float*>(smem);
    float* mac = reinterpret_cast<float*>(smem + C::OFF_MAC); // rho, ux, uy, T [4][MWB]
    unsigned char* ign = smem + C::OFF_IGN;
    float* par = reinterpret_cast<float*>(smem + C::OFF_PAR); // S[16], A8c, A9c, chem, om1, om2
    const int tid = threadIdx.x;
    const int lx = 2 * tid + 4, mi = 2 * tid + 2;
    const DfConst Cd = df_constants(K);
    const float dt = K.dt;
    const unsigned expected = gridDim.x + (unsigned)b.phantom_blocks;
    int bad = 0;

    for (int s = 0; s < b.nsteps; s++) {
        const float* __restrict__ in = static_cast<const float*>(b.buf[(b.cur + s) & 1]);
        float* __restrict__ out = static_cast<float*>(b.buf[(b.cur + s + 1) & 1]);
        int cb = 0;
        int item = blockIdx.x;
        if (item < b.nitems) {
            const BatchItem it = b.items[item];
            stage_item<BT>(in, stage, b.inst[it.inst], it.x0, K.plane);
        }
        cp_commit();
        for (; item < b.nitems; item += gridDim.x) {
            const int nxt = item + gridDim.x;
            if (nxt < b.nitems) {
                const BatchItem it2 = b.items[nxt];
                stage_item<BT>(in, stage + (cb ^ 1) * NPLANE * C::SW, b.inst[it2.inst], it2.x0,
                               K.plane);
            }
            cp_commit();
            const BatchItem it = b.items[item];
            const InstParam& ip = b.inst[it.inst];
            if (tid < 16) par[tid] = ip.S[tid];
            if (tid == 16) par[16] = ip.A8c;
            if (tid == 17) par[17] = ip.A9c;
            if (tid == 18) par[18] = ip.chem;
            if (tid == 19) par[19] = ip.om1;
            if (tid == 20) par[20] = ip.om2;
            cp_wait<1>();
            __syncthreads();
            const float* sb = stage + cb * NPLANE * C::SW;
            const int cx = it.x0 + 2 * tid;
            const bool act0 = cx < ip.nx, act1 = cx + 1 < ip.nx;

            // rho, u, T of the two cells (conserved moments, Eqs. (5)-(7)) and halo u
            {
                V2 f[16];
#pragma unroll
                for (int i = 0; i < 16; i++) f[i] = ldv(sb + i * C::SW + lx);
                V2 rho, ux, uy, T;
                bool ig0, ig1, ok0, ok1;
                recover_pair_fast<REC>(f, Cd, K, rho, ux, uy, T, ig0, ig1, ok0, ok1);
                if ((act0 && !ok0) || (act1 && !ok1)) bad = 1;
                *reinterpret_cast<float2*>(mac + 0 * C::MWB + mi) = rho.v;
                *reinterpret_cast<float2*>(mac + 1 * C::MWB + mi) = ux.v;
                *reinterpret_cast<float2*>(mac + 2 * C::MWB + mi) = uy.v;
                *reinterpret_cast<float2*>(mac + 3 * C::MWB + mi) = T.v;
                ign[2 * tid] = ig0;
                ign[2 * tid + 1] = ig1;
                if (tid == 0 || tid == BT - 1) {
                    const int hx = tid == 0 ? 3 : C::SEG + 4;
                    const int hm = tid == 0 ? 1 : C::SEG + 2;
                    float g[16];
#pragma unroll
                    for (int i = 0; i < 16; i++) g[i] = sb[i * C::SW + hx];
                    float hu, hv;
                    velocity_f32(g, K, hu, hv);
                    mac[1 * C::MWB + hm] = hu;
                    mac[2 * C::MWB + hm] = hv;
                }
            }
            __syncthreads();

            // update of the two cells
            {
                V2 f[16];
#pragma unroll
                for (int i = 0; i < 16; i++) f[i] = ldv(sb + i * C::SW + lx);
                const V2 lam0 = ldv(sb + 16 * C::SW + lx);
                const V2 rho = ldv(mac + 0 * C::MWB + mi), ux = ldv(mac + 1 * C::MWB + mi);
                const V2 uy = ldv(mac + 2 * C::MWB + mi), T = ldv(mac + 3 * C::MWB + mi);
                V2 m[16], q[16], D[TNE_K];
                forward_moments(K, f, m);
                feq_moments(V2(K.DI), rho, ux, uy, T, q);
#pragma unroll
                for (int k = 0; k < TNE_K; k++) D[k] = m[k + 4] - q[k + 4];
                const float2 uxl = *reinterpret_cast<const float2*>(mac + 1 * C::MWB + mi - 2);
                const float2 uxh = *reinterpret_cast<const float2*>(mac + 1 * C::MWB + mi + 2);
                const float2 uyl = *reinterpret_cast<const float2*>(mac + 2 * C::MWB + mi - 2);
                const float2 uyh = *reinterpret_cast<const float2*>(mac + 2 * C::MWB + mi + 2);
                const V2 dux_dx = (V2(ux.y(), uxh.x) - V2(uxl.y, ux.x())) * K.half_inv_dx;
                const V2 duy_dx = (V2(uy.y(), uyh.x) - V2(uyl.y, uy.x())) * K.half_inv_dx;
                const V2 theta = dux_dx * K.inv_DI;
                const V2 rT = rho * T;
                const V2 A8 = (rT * par[16]) * fma(V2(4.f) * ux, dux_dx - theta, V2(2.f) * uy * duy_dx);
                const V2 A9 = (rT * par[17]) * fma(V2(4.f) * uy, -theta, V2(2.f) * ux * duy_dx);
                // both cells evaluated, then selected: no divergent branch
                const float ri0 = reaction_increment(lam0.x(), par[19] * rT.x(), par[20] * rT.x(), dt);
                const float ri1 = reaction_increment(lam0.y(), par[19] * rT.y(), par[20] * rT.y(), dt);
                const float dl0 = ign[2 * tid] ? ri0 : 0.f, dl1 = ign[2 * tid + 1] ? ri1 : 0.f;
                const V2 dlam(dl0, dl1);
                const V2 cr = dlam * par[18];
                V2 dq[16], Om[16], W[16];
                dfeq_dT(V2(K.DI), rho, ux, uy, T, dq);
                Om[0] = Om[1] = Om[2] = V2(0.f);
                Om[3] = dq[3] * cr;
#pragma unroll
                for (int k = 4; k < 16; k++) Om[k] = fma(V2(-par[k]), D[k - 4], dq[k] * cr);
                Om[7] += A8;
                Om[8] += A9;
                inverse_moments(K, Om, W);

                const Q6 lq = load6(sb + 16 * C::SW, lx);
                const V2 lpx = nnd_pos_x(lq), lnx = nnd_neg_x(lq);
                const V2 lax(ux.x() > 0.f ? lpx.x() : lnx.x(), ux.y() > 0.f ? lpx.y() : lnx.y());
                V2 ln = fma(V2(-dt), ux * K.inv_dx * lax, lam0) + dlam;
                ln = vmin(vmax(ln, V2(0.f)), V2(1.f));

                const int64_t g = ip.off + cx;
                auto put = [&](int i, V2 adv) {
                    const V2 v = fma(V2(dt), W[i] - adv, f[i]);
                    if (act1)
                        *reinterpret_cast<float2*>(out + i * K.plane + g) = v.v;
                    else if (act0)
                        out[i * K.plane + g] = v.x();
                };
#define PX(i) nnd_pos_x(load6(sb + (i) * C::SW, lx))
#define NX(i) nnd_neg_x(load6(sb + (i) * C::SW, lx))
#pragma unroll
                for (int o = 0; o < 2; o++) { // axis orbits: only (+-c, 0) move along x
                    const int i0 = 8 * o;
                    const float cxs = K.c[2 * o] * K.inv_dx;
                    put(i0 + 0, cxs * PX(i0 + 0));
                    put(i0 + 1, V2(0.f));
                    put(i0 + 2, -cxs * NX(i0 + 2));
                    put(i0 + 3, V2(0.f));
                }
#pragma unroll
                for (int o = 0; o < 2; o++) { // diagonal orbits
                    const int i0 = 4 + 8 * o;
                    const float cxs = K.c[2 * o + 1] * K.inv_dx;
                    put(i0 + 0, cxs * PX(i0 + 0));
                    put(i0 + 1, -cxs * NX(i0 + 1));
                    put(i0 + 2, -cxs * NX(i0 + 2));
                    put(i0 + 3, cxs * PX(i0 + 3));
                }
#undef PX
#undef NX
                if (act1)
                    *reinterpret_cast<float2*>(out + 16 * K.plane + g) = ln.v;
                else if (act0)
                    out[16 * K.plane + g] = ln.x();
            }
            __syncthreads(); // the staging buffer and macro row are reused
            cb ^= 1;
        }
        cp_wait<0>();
        if (__syncthreads_or(bad) && tid == 0) atomicOr(&b.ctr->status, 1);
        bad = 0;
        if (!grid_barrier(b, expected)) return;
        if (blockIdx.x == 0 && tid == 0) b.ctr->step += 1;
    }
}

template <int REC, int BT>
cudaError_t batch_prepare()
{
    static cudaError_t done = cudaFuncSetAttribute(
        batch_kernel<REC, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BCfg<BT>::SMEM);
    return done;
}

template <int REC, int BT>
int batch_max_blocks_per_sm()
{
    if (batch_prepare<REC, BT>() != cudaSuccess) return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<REC, BT>, BT,
                                                      BCfg<BT>::SMEM) != cudaSuccess)
        return -1;
    return per_sm;
}

template <int REC, int BT>
cudaError_t batch_launch_t(const ModelConst<float>& K, const BatchLaunch& b, int grid,
                           cudaStream_t s)
{
    cudaError_t e = batch_prepare<REC, BT>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = BCfg<BT>::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<REC, BT>, K, b);
}

constexpr int TI_THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(TI_THREADS)
    tne_instances_kernel(const ModelConst<double> K, const R* state, const InstParam* inst,
                         TneRecord* out, double area)
{
    __shared__ double ssum[TI_THREADS / 32][2 * TNE_K + 2];
    __shared__ double smn[TI_THREADS / 32][TNE_K], smx[TI_THREADS / 32][TNE_K];
    const InstParam& ip = inst[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[2 * TNE_K + 2], mn[TNE_K], mx[TNE_K];
    for (int q = 0; q < 2 * TNE_K + 2; q++) acc[q] = 0.0;
    for (int k = 0; k < TNE_K; k++) mn[k] = DBL_MAX, mx[k] = -DBL_MAX;
    for (int x = threadIdx.x; x < ip.nx; x += TI_THREADS) {
        const int64_t g = ip.off + x;
        double f[16], m[16], q[16];
        for (int i = 0; i < 16; i++) f[i] = (double)state[i * K.plane + g];
        forward_moments(K, f, m);
        const double r = m[0], u = m[1] / r, v = m[2] / r;
        const double t = (m[3] / r - (u * u + v * v)) * K.inv_DId;
        feq_moments(K.DI, r, u, v, t, q);
        double d2 = 0.0;
        for (int k = 4; k < 16; k++) {
            const double D = m[k] - q[k];
            acc[k - 4] += D;
            acc[TNE_K + k - 4] += fabs(D);
            mn[k - 4] = fmin(mn[k - 4], D);
            mx[k - 4] = fmax(mx[k - 4], D);
            d2 += D * D;
        }
        acc[2 * TNE_K] += sqrt(d2);
        acc[2 * TNE_K + 1] += d2;
    }
    for (int q = 0; q < 2 * TNE_K + 2; q++) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) ssum[warp][q] = v;
    }
    for (int k = 0; k < TNE_K; k++) {
        double a = mn[k], c = mx[k];
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
        }
        if (lane == 0) smn[warp][k] = a, smx[warp][k] = c;
    }
    __syncthreads();
    TneRecord* rec = out + blockIdx.x;
    const int k = threadIdx.x;
    if (k < 16) {
        double s0 = 0, s1 = 0, a = DBL_MAX, c = -DBL_MAX;
        if (k >= 4)
            for (int w = 0; w < TI_THREADS / 32; w++) {
                s0 += ssum[w][k - 4];
                s1 += ssum[w][TNE_K + k - 4];
                a = fmin(a, smn[w][k - 4]);
                c = fmax(c, smx[w][k - 4]);
            }
        rec->sum[k] = k < 4 ? 0.0 : s0 * area;
        rec->abs_sum[k] = k < 4 ? 0.0 : s1 * area;
        rec->min[k] = k < 4 ? 0.0 : a;
        rec->max[k] = k < 4 ? 0.0 : c;
    } else if (k == 32) {
        double d = 0, d2 = 0;
        for (int w = 0; w < TI_THREADS / 32; w++) d += ssum[w][2 * TNE_K], d2 += ssum[w][2 * TNE_K + 1];
        rec->d_sum = d * area;
        rec->d2_sum = d2 * area;
        rec->step = -1;
    }
}

} // namespace

cudaError_t launch_tne_instances(int precision, const ModelConst<double>& Kd, const void* state,
                                 const InstParam* inst, int n_inst, TneRecord* out,
                                 double area, cudaStream_t s)
{
    if (precision == 0)
        tne_instances_kernel<double><<<n_inst, TI_THREADS, 0, s>>>(
            Kd, static_cast<const double*>(state), inst, out, area);
    else
        tne_instances_kernel<float><<<n_inst, TI_THREADS, 0, s>>>(
            Kd, static_cast<const float*>(state), inst, out, area);
    return cudaGetLastError();
}

int batch_segment(int block_threads) { return 2 * block_threads; }

int batch_max_blocks(int recovery, int block_threads)
{
    if (block_threads == 64)
        return recovery == 1 ? batch_max_blocks_per_sm<1, 64>() : batch_max_blocks_per_sm<0, 64>();
    if (block_threads == 128)
        return recovery == 1 ? batch_max_blocks_per_sm<1, 128>() : batch_max_blocks_per_sm<0, 128>();
    return -1;
}

cudaError_t launch_batch(int recovery, int block_threads, const ModelConst<float>& K,
                         const BatchLaunch& b, int grid, cudaStream_t s)
{
    if (block_threads == 64)
        return recovery == 1 ? batch_launch_t<1, 64>(K, b, grid, s) : batch_launch_t<0, 64>(K, b, grid, s);
    if (block_threads == 128)
        return recovery == 1 ? batch_launch_t<1, 128>(K, b, grid, s)
                             : batch_launch_t<0, 128>(K, b, grid, s);
    return cudaErrorInvalidValue;
}

} // namespace lbk
