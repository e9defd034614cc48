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
// Combining them is latency-bound (they sit in L2), so every thread of the finishing
// block walks its own blocks (t, t + T, ...) for ten quantities at a time with twenty
// loads in flight, then the lanes combine in a fixed shuffle tree and the warps in
// warp order: deterministic for a given grid.
__device__ __forceinline__ double tne_comb(int kind, double a, double b)
{
    return kind == 0 ? a + b : (kind == 1 ? fmin(a, b) : fmax(a, b));
}
__device__ __forceinline__ int tne_kind(int q)
{
    return (q < 2 * TNE_K || q >= 4 * TNE_K) ? 0 : (q < 3 * TNE_K ? 1 : 2);
}
static __device__ __noinline__ void finish_tne(const double* partials, int nblocks, TneRecord* rec,
                                               int64_t step, double area)
{
    constexpr int QC = 10;
    static_assert(TNE_PART % QC == 0, "quantities in chunks of ten");
    __shared__ double res[TNE_PART];
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5, nw = T >> 5;
    for (int q0 = 0; q0 < TNE_PART; q0 += QC) {
        double acc[QC];
#pragma unroll
        for (int k = 0; k < QC; k++) {
            const int kind = tne_kind(q0 + k);
            acc[k] = kind == 0 ? 0.0 : (kind == 1 ? DBL_MAX : -DBL_MAX);
        }
        int b = t;
        for (; b + T < nblocks; b += 2 * T) {
            double v0[QC], v1[QC];
#pragma unroll
            for (int k = 0; k < QC; k++) {
                v0[k] = __ldcg(partials + (size_t)(q0 + k) * nblocks + b);
                v1[k] = __ldcg(partials + (size_t)(q0 + k) * nblocks + b + T);
            }
#pragma unroll
            for (int k = 0; k < QC; k++) {
                const int kind = tne_kind(q0 + k);
                acc[k] = tne_comb(kind, tne_comb(kind, acc[k], v0[k]), v1[k]);
            }
        }
        if (b < nblocks) {
#pragma unroll
            for (int k = 0; k < QC; k++)
                acc[k] = tne_comb(tne_kind(q0 + k), acc[k],
                                  __ldcg(partials + (size_t)(q0 + k) * nblocks + b));
        }
#pragma unroll
        for (int k = 0; k < QC; k++) {
            const int kind = tne_kind(q0 + k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                acc[k] = tne_comb(kind, acc[k], __shfl_xor_sync(0xffffffffu, acc[k], o));
        }
        for (int ww = 0; ww < nw; ww++) {
            if (w == ww && lane == 0) {
#pragma unroll
                for (int k = 0; k < QC; k++)
                    res[q0 + k] = ww == 0 ? acc[k] : tne_comb(tne_kind(q0 + k), res[q0 + k], acc[k]);
            }
            __syncthreads();
        }
    }
    for (int k = t; k < 16; k += T) {
        const bool z = k < 4;
        rec->sum[k] = z ? 0.0 : res[k - 4] * area;
        rec->abs_sum[k] = z ? 0.0 : res[TNE_K + k - 4] * area;
        rec->min[k] = z ? 0.0 : res[2 * TNE_K + k - 4];
        rec->max[k] = z ? 0.0 : res[3 * TNE_K + k - 4];
    }
    if (t == 0) {
        rec->d_sum = res[4 * TNE_K] * area;
        rec->d2_sum = res[4 * TNE_K + 1] * area;
        rec->step = step;
    }
}


} // namespace lbk
