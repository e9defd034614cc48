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
static __device__ __noinline__ void finish_tne(const double* partials, int nblocks, TneRecord* rec, int64_t step,
                           double area)
{
    __shared__ double res[TNE_PART];
    for (int q = threadIdx.x; q < TNE_PART; q += blockDim.x) {
        double acc;
        if (q < 2 * TNE_K || q >= 4 * TNE_K) {
            acc = 0.0;
            for (int b = 0; b < nblocks; b++) acc += __ldcg(partials + (size_t)b * TNE_PART + q);
            acc *= area;
        } else if (q < 3 * TNE_K) {
            acc = DBL_MAX;
            for (int b = 0; b < nblocks; b++)
                acc = fmin(acc, __ldcg(partials + (size_t)b * TNE_PART + q));
        } else {
            acc = -DBL_MAX;
            for (int b = 0; b < nblocks; b++)
                acc = fmax(acc, __ldcg(partials + (size_t)b * TNE_PART + q));
        }
        res[q] = acc;
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
