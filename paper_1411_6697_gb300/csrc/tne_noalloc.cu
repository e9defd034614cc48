// tne_noalloc.cu -- grid-wide TNE measures of a caller-owned state without any
// device allocation (lbkm_tne_noalloc in include/lbkm.h).
//
// Some callers cannot allocate device memory: an application whose own pool
// already holds the whole device memory, or a latency-bound loop that must not
// pay the implicit device-wide synchronisation of cudaMalloc/cudaFree. For
// them this entry point needs no handle and allocates nothing: the caller
// passes the state and the output, and the per-block partial sums and the
// arrival counter live in the file-scope device arrays below. Every GPU that
// loads the library holds these arrays (about 0.8 MB) until the process exits.
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>

#include "lbkm.h"
#include "cell.cuh"
#include "kernels.cuh"
#include "model.h"

namespace lbk {

void set_handleless_error(const char* msg);

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_BLOCK = NA_THREADS * 32;
constexpr int NA_MAX_BLOCKS = 2048; // => at most 2048 * 8192 = 16,777,216 cells (4096 x 4096)
constexpr int NA_SUMS = 2 * TNE_K + 2;

// Shared by every call on a device; the last call's contents stay behind.
static __device__ __align__(256) double g_na_partials[NA_MAX_BLOCKS * TNE_PART];
static __device__ __align__(256) unsigned int g_na_arrivals;

// Device addresses of the two arrays, per device ordinal, as the last lookup on that
// device found them. Calls outside stream capture look them up again (a device reset
// or a new primary context moves them); calls during capture use the stored value.
constexpr int NA_MAX_DEVICES = 64;
std::atomic<uintptr_t> g_partials_addr[NA_MAX_DEVICES];
std::atomic<uintptr_t> g_arrivals_addr[NA_MAX_DEVICES];

__device__ __forceinline__ double na_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double na_warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double na_warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block b reduces cells [b * NA_CELLS_PER_BLOCK, (b + 1) * NA_CELLS_PER_BLOCK); the last
// block to finish combines the partials in block order and writes the record.
template <typename R>
__global__ void __launch_bounds__(NA_THREADS)
    tne_noalloc_kernel(const ModelConst<double> K, const R* state, int64_t pitch, double* delta,
                       double* partials, unsigned int* arrivals, TneRecord* out, double area)
{
    __shared__ double ssum[NA_THREADS / 32][NA_SUMS];
    __shared__ double smm[NA_THREADS / 32][2 * TNE_K];
    __shared__ double res[TNE_PART];
    __shared__ unsigned int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[NA_SUMS], mn[TNE_K], mx[TNE_K];
    for (int q = 0; q < NA_SUMS; q++) acc[q] = 0.0;
    for (int k = 0; k < TNE_K; k++) mn[k] = DBL_MAX, mx[k] = -DBL_MAX;
    const int64_t n = (int64_t)K.nx * K.ny;
    const int64_t plane = (int64_t)K.ny * pitch;
    const int64_t c0 = (int64_t)blockIdx.x * NA_CELLS_PER_BLOCK;
    const int64_t c1 = c0 + NA_CELLS_PER_BLOCK < n ? c0 + NA_CELLS_PER_BLOCK : n;
    for (int64_t c = c0 + threadIdx.x; c < c1; c += NA_THREADS) {
        const int y = (int)(c / K.nx), x = (int)(c - (int64_t)y * K.nx);
        const int64_t g = (int64_t)y * pitch + x;
        double f[16], m[16], q[16];
        for (int i = 0; i < 16; i++) f[i] = (double)state[i * plane + g];
        forward_moments(K, f, m);
        const double r = m[0], u = m[1] / r, v = m[2] / r;
        const double t = (m[3] / r - (u * u + v * v)) * K.inv_DId;
        feq_moments(K.DI, r, u, v, t, q);
        double d2 = 0.0;
        for (int k = 0; k < 16; k++) {
            const double D = k < 4 ? 0.0 : m[k] - q[k];
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
    for (int q = 0; q < NA_SUMS; q++) {
        const double s = na_warp_sum(acc[q]);
        if (lane == 0) ssum[warp][q] = s;
    }
    for (int k = 0; k < TNE_K; k++) {
        const double a = na_warp_min(mn[k]), b = na_warp_max(mx[k]);
        if (lane == 0) smm[warp][k] = a, smm[warp][TNE_K + k] = b;
    }
    __syncthreads();
    double* part = partials + (size_t)blockIdx.x * TNE_PART;
    if (threadIdx.x < NA_SUMS) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++) s += ssum[w][threadIdx.x];
        const int q = threadIdx.x;
        part[q < 2 * TNE_K ? q : 4 * TNE_K + (q - 2 * TNE_K)] = s;
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + 2 * TNE_K) {
        const int q = threadIdx.x - 32;
        double v = smm[0][q];
        for (int w = 1; w < NA_THREADS / 32; w++)
            v = q < TNE_K ? fmin(v, smm[w][q]) : fmax(v, smm[w][q]);
        part[2 * TNE_K + q] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(arrivals, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < TNE_PART; q += NA_THREADS) {
        double a;
        if (q < 2 * TNE_K || q >= 4 * TNE_K) {
            a = 0.0;
            for (unsigned b = 0; b < gridDim.x; b++) a += __ldcg(partials + (size_t)b * TNE_PART + q);
            a *= area;
        } else if (q < 3 * TNE_K) {
            a = DBL_MAX;
            for (unsigned b = 0; b < gridDim.x; b++)
                a = fmin(a, __ldcg(partials + (size_t)b * TNE_PART + q));
        } else {
            a = -DBL_MAX;
            for (unsigned b = 0; b < gridDim.x; b++)
                a = fmax(a, __ldcg(partials + (size_t)b * TNE_PART + q));
        }
        res[q] = a;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 16; k += NA_THREADS) {
        const bool z = k < 4;
        out->sum[k] = z ? 0.0 : res[k - 4];
        out->abs_sum[k] = z ? 0.0 : res[TNE_K + k - 4];
        out->min[k] = z ? 0.0 : res[2 * TNE_K + k - 4];
        out->max[k] = z ? 0.0 : res[3 * TNE_K + k - 4];
    }
    if (threadIdx.x == 0) {
        out->d_sum = res[4 * TNE_K];
        out->d2_sum = res[4 * TNE_K + 1];
        out->step = -1;
        *arrivals = 0u;
    }
}

lbkm_status na_fail(lbkm_status st, const char* msg)
{
    set_handleless_error(msg);
    return st;
}

} // namespace
} // namespace lbk

using namespace lbk;

extern "C" lbkm_status lbkm_tne_noalloc(const lbkm_params* p, const void* state, int64_t pitch,
                                        double* delta, lbkm_tne_global* out, void* cuda_stream)
{
    if (!p || !state || !out) return na_fail(LBKM_EINVAL, "params, state and out are required");
    if (p->nx < 1 || p->ny < 1) return na_fail(LBKM_EINVAL, "nx and ny must be >= 1");
    if (pitch < p->nx) return na_fail(LBKM_EINVAL, "pitch must be >= nx");
    if (pitch > INT_MAX) return na_fail(LBKM_EINVAL, "pitch must be <= 2147483647 elements");
    if (p->precision != LBKM_F64 && p->precision != LBKM_F32)
        return na_fail(LBKM_EINVAL, "precision must be LBKM_F64 or LBKM_F32");
    if (!(p->gamma > 1.0 && p->gamma <= 2.0))
        return na_fail(LBKM_EINVAL, "gamma must lie in (1, 2]");
    const int64_t n = (int64_t)p->nx * p->ny;
    const int64_t blocks = (n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK;
    if (blocks > NA_MAX_BLOCKS) {
        char m[200];
        snprintf(m, sizeof(m),
                 "lbkm_tne_noalloc handles at most %d cells (fixed scratch); got %lld",
                 NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK, (long long)n);
        return na_fail(LBKM_EINVAL, m);
    }
    HostModel hm;
    char err[256] = {0};
    if (build_host_model(p->orbit_kind, p->orbit_speed, p->orbit_eta, p->gamma, &hm, err,
                         sizeof(err)) != 0)
        return na_fail(strstr(err, "orbit_kind") ? LBKM_EINVAL : LBKM_ESINGULAR, err);
    ModelConst<double> K;
    fill_model_const<double>(hm, p->S, p->Q, p->omega1, p->omega2, p->T_ig, p->dx, p->dy, p->dt,
                             p->nx, p->ny, (int)pitch, p->bc_x, p->bc_y, &K);

    // device addresses of the file-scope scratch (the names are host-side stand-ins in
    // host code), looked up with the calling device current
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(LBKM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(LBKM_EINVAL, "device ordinal too large");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return na_fail(LBKM_ECUDA, cudaGetErrorString(e));
    if (cap == cudaStreamCaptureStatusNone) {
        void* a = nullptr;
        void* b = nullptr;
        e = cudaGetSymbolAddress(&a, g_na_partials);
        if (e != cudaSuccess) return na_fail(LBKM_ECUDA, cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&b, g_na_arrivals);
        if (e != cudaSuccess) return na_fail(LBKM_ECUDA, cudaGetErrorString(e));
        g_partials_addr[dev].store(reinterpret_cast<uintptr_t>(a), std::memory_order_release);
        g_arrivals_addr[dev].store(reinterpret_cast<uintptr_t>(b), std::memory_order_release);
    }
    double* partials = reinterpret_cast<double*>(g_partials_addr[dev].load(std::memory_order_acquire));
    unsigned int* arrivals =
        reinterpret_cast<unsigned int*>(g_arrivals_addr[dev].load(std::memory_order_acquire));
    if (!partials || !arrivals)
        return na_fail(LBKM_ESTATE, "lbkm_tne_noalloc: the first call on a device must come "
                                    "before any stream capture");
    // the arrival counter must start at zero whatever an earlier call left behind
    e = cudaMemsetAsync(arrivals, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return na_fail(LBKM_ECUDA, cudaGetErrorString(e));
    TneRecord* o = reinterpret_cast<TneRecord*>(out);
    const double area = p->dx * p->dy;
    if (p->precision == LBKM_F64)
        tne_noalloc_kernel<double><<<(unsigned)blocks, NA_THREADS, 0, s>>>(
            K, static_cast<const double*>(state), pitch, delta, partials, arrivals, o, area);
    else
        tne_noalloc_kernel<float><<<(unsigned)blocks, NA_THREADS, 0, s>>>(
            K, static_cast<const float*>(state), pitch, delta, partials, arrivals, o, area);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(LBKM_ECUDA, cudaGetErrorString(e));
    return LBKM_OK;
}
