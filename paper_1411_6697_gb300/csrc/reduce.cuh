// reduce.cuh -- warp reductions and the deterministic finish of the grid-wide
// TNE record shared by the step kernels.
#pragma once
#include <float.h>

#include "cell.cuh"
#include "kernels.cuh"

namespace lbk {

constexpr int NSUM = 2 * TNE_K + 2; // sums: Delta, |Delta|, d, d^2
constexpr int NMM = 2 * TNE_K;      // min, max


template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R>
__device__ __forceinline__ R warp_min(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = rmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename R>
__device__ __forceinline__ R warp_max(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = rmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename R>
__device__ __forceinline__ R big_value();
template <>
__device__ __forceinline__ float big_value<float>() { return FLT_MAX; }
template <>
__device__ __forceinline__ double big_value<double>() { return DBL_MAX; }

// Last block of a launch: reduce the per-block partials (fixed order) into a
// TNE record. Called by every thread of that block.
// Partials are stored quantity-major: partial q of block b at partials[q * nblocks + b].
// Each quantity is reduced by one warp: lane l combines blocks l, l+32, ... in
// order, then the lanes combine in a fixed shuffle tree (deterministic).
static __device__ __noinline__ void finish_tne(const double* partials, int nblocks, TneRecord* rec,
                                               int64_t step, double area)
{
    __shared__ double res[TNE_PART];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = threadIdx.x >> 5; q < TNE_PART; q += nw) {
        const double* pq = partials + (size_t)q * nblocks;
        const int kind = (q < 2 * TNE_K || q >= 4 * TNE_K) ? 0 : (q < 3 * TNE_K ? 1 : 2);
        double acc = kind == 0 ? 0.0 : (kind == 1 ? DBL_MAX : -DBL_MAX);
        for (int b = lane; b < nblocks; b += 32) {
            const double v = __ldcg(pq + b);
            acc = kind == 0 ? acc + v : (kind == 1 ? fmin(acc, v) : fmax(acc, v));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = kind == 0 ? acc + v : (kind == 1 ? fmin(acc, v) : fmax(acc, v));
        }
        if (lane == 0) res[q] = kind == 0 ? acc * area : acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 16; k += blockDim.x) {
        bool z = k < 4;
        rec->sum[k] = z ? 0.0 : res[k - 4];
        rec->abs_sum[k] = z ? 0.0 : res[TNE_K + k - 4];
        rec->min[k] = z ? 0.0 : res[2 * TNE_K + k - 4];
        rec->max[k] = z ? 0.0 : res[3 * TNE_K + k - 4];
    }
    if (threadIdx.x == 0) {
        rec->d_sum = res[4 * TNE_K];
        rec->d2_sum = res[4 * TNE_K + 1];
        rec->step = step;
    }
}


} // namespace lbk
