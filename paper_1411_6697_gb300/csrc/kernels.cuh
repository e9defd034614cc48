// kernels.cuh -- launch interface between the C ABI and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "model.h"

namespace lbk {

// Device-side bookkeeping shared by the kernels of one handle.
struct DevCounters {
    int64_t step;          // steps taken (advanced by the last block of each step)
    int64_t hist_count;    // TNE records written so far
    unsigned int arrivals; // blocks of the current launch that finished (reset by the last)
    int status;            // bit 0: non-finite or non-positive rho or T seen
    int tne_pending;       // the launch just finished left TNE partials (set every step)
    int pad;
    int64_t tne_step;      // step index of those partials
};

// One on-the-fly TNE record, laid out like lbkm_tne_global.
struct TneRecord {
    double sum[16], abs_sum[16], min[16], max[16];
    double d_sum, d2_sum;
    int64_t step;
};

// An encoded TMA tensor map (the driver's opaque 128-byte CUtensorMap).
struct alignas(64) TmaDesc {
    unsigned long long w[16];
};

struct StepLaunch {
    const void* in;      // state at t_n  [17][ny][pitch]
    void* out;           // state at t_n+1
    // stage: 0 forward Euler step; 1 first stage of an SSP Runge-Kutta step (writes
    // E(u^n), reduces the TNE of u^n, does not advance the step counter); 2 last stage
    // (writes wprev * prev + wnew * E(in) with prev = u^n, no TNE, advances the
    // counter); 3 a middle stage (the same weighted write, no TNE, no counter)
    const void* prev;
    int stage;
    double wprev, wnew;
    double* partials;    // [grid][TNE_PART]
    DevCounters* ctr;
    TneRecord* hist;     // ring of hist_cap records
    int hist_cap;
    int tne_every;       // 0 = off
    int grid;            // blocks launched
    double cell_area;    // dx * dy
    const TmaDesc* tm_in;  // host copies of the tensor maps of in (loads) and out (stores),
    const TmaDesc* tm_out; // FP32 2-D grids only
    int srt;               // 1: single-relaxation-time collision (equal rates, no TNE)
};

// Grid-wide TNE record of the partials a step left (if its schedule reduced TNE): one
// block per quantity, each a fixed-order reduction over the step's blocks, written into
// history slot (hist_count - 1) % hist_cap. Launched after every full step.
cudaError_t launch_tne_finish(const StepLaunch& a, cudaStream_t s);

// precision: 0 = FP64, 1 = FP32; recovery: 0 = FP64, 1 = double-float (FP32 only)
cudaError_t launch_step(int precision, int recovery, bool two_d, const void* K,
                        const StepLaunch& a, cudaStream_t s);
// Blocks to launch for a step on this grid (multiple of the SM count times the
// resident blocks per SM, capped by the number of tiles).
// sbc: the side conditions (walls, Dirichlet or specular sides select the general
// variant of the FP32 marching kernel)
int step_grid(int precision, int recovery, bool two_d, int nx, int ny, const int sbc[4]);

cudaError_t launch_init(int precision, const ModelConst<double>& Kd, const double* rho,
                        const double* ux, const double* uy, const double* T, const double* lam,
                        void* state, cudaStream_t s);
cudaError_t launch_macros(int precision, const ModelConst<double>& Kd, const void* state,
                          double* rho, double* ux, double* uy, double* T, double* p,
                          double* lam, cudaStream_t s);
// TNE fields (optional) and grid-wide record of a state, all FP64.
cudaError_t launch_tne(int precision, const ModelConst<double>& Kd, const void* state,
                       double* delta, double* partials, int grid, DevCounters* ctr,
                       TneRecord* out, double cell_area, cudaStream_t s);
int tne_grid(int nx, int ny);

// Batched 1-D instances (batch.cu): per-instance parameters, work items and the
// arguments of one persistent launch.
struct InstParam {
    float S[16];
    float A8c, A9c, chem, om1, om2; // (S5-S8)/S5, (S7-S9)/S7, 2Q/((D+I)dt), omega1, omega2
    int32_t nx;
    int64_t off; // first cell of the instance in the flat layout
};
struct BatchItem {
    int32_t inst, x0; // instance and first cell of the segment
};
struct BatchLaunch {
    void* buf[2];
    int cur;             // buffer holding the input of the first step
    const InstParam* inst;
    const BatchItem* items;
    int nitems;
    DevCounters* ctr;
    unsigned* bar;       // grid barrier: arrivals, generation
    int nsteps;
    int phantom_blocks;  // > 0 only to test the bounded barrier wait
    long long wait_ns;   // bound of each barrier wait
};
int batch_segment(int block_threads);
int batch_max_blocks(int recovery, int block_threads);
cudaError_t launch_batch(int recovery, int block_threads, const ModelConst<float>& K,
                         const BatchLaunch& b, int grid, cudaStream_t s);
// grid-wide TNE record of every instance (one block per instance, FP64)
cudaError_t launch_tne_instances(int precision, const ModelConst<double>& Kd, const void* state,
                                 const InstParam* inst, int n_inst, TneRecord* out,
                                 double area, cudaStream_t s);

// Discrete adjoint of the FP64 1-D step (adjoint.cu).
constexpr int ADJ_NPAR = 15; // dJ/dS_5..S_16, dJ/dQ, dJ/domega1, dJ/domega2
struct AdjArgs {
    const double* f;     // state n: 17 planes with the handle's pitch
    const double* mac;   // [4][nx] rho, ux, uy, T of state n
    const double* fb1;   // dJ/df of state n+1, [16][nx]
    const double* lb1;   // dJ/dlambda of state n+1, [nx]
    double* mb;          // [16][nx] pass A -> B: adjoint of the moments
    double* loc;         // [6][nx] pass A -> B: rho_b, ux_b, uy_b, T_b, lambda_b, clamped lambda_b
    double* gb;          // [2][nx] pass A -> B: adjoints of du_x/dx, du_y/dx
    double* cw;          // [17][5][nx] pass A -> B: weighted NND coefficients of each cell's
                         // stencil (planes f_1..f_16, lambda; offsets -2..+2)
    double* fb0;         // dJ/df of state n, [16][nx]
    double* lb0;         // dJ/dlambda of state n, [nx]
    double* pacc;        // [ADJ_NPAR][grid] per-block parameter accumulators
    double* jacc;        // [grid] per-block objective accumulators
    const double* vx;    // [16] x-velocities (M, M^-1 and their transposes act in block form)
    double tne_w;        // w_tne dx dt: Delta_b += 2 tne_w Delta
    double jw;           // w_tne dx dt for the objective value
};
int adj_grid(int nx);
cudaError_t launch_adj_step(const ModelConst<double>& K, const AdjArgs& a, int grid,
                            cudaStream_t s);
cudaError_t launch_adj_seed(const ModelConst<double>& K, const AdjArgs& a, const double* rho_t,
                            double w, int grid, cudaStream_t s);
cudaError_t launch_adj_rho0(const ModelConst<double>& K, const AdjArgs& a, double* drho0,
                            int grid, cudaStream_t s);
// n floats widened to doubles (an FP32 forward run's checkpoint, to restart a segment in FP64)
cudaError_t launch_adj_widen(const float* in, double* out, size_t n, int grid, cudaStream_t s);

// FP32 2-D step: y-marching strips, two cells per thread (march.cu)
// mode = recovery | (general side conditions << 1)
// Tensor maps of an FP32 state buffer for the step kernel's bulk tensor copies: loads of
// a box of BW + 8 columns x 2 rows x 17 planes, stores of BW x 2 x 17.
cudaError_t march_tensor_maps(const void* state, int nx, int ny, int pitch, int64_t plane,
                              TmaDesc* load, TmaDesc* store);
int march_grid(int mode, int nx, int ny);
cudaError_t launch_march(int mode, const ModelConst<float>& K, const StepLaunch& a,
                         cudaStream_t s);

} // namespace lbk
