// The objective of the discrete adjoint without its derivative (adjoint.cu).
#pragma once
#include "kernels.cuh"

namespace lbk {

// Adds w_tne dx dt sum_x d^2 of the FP64 state a.f (d^2 = sum_{k=5..16} Delta_k^2,
// Sec. VI, Eq. (91); rho, u, T recovered in the kernel) to the per-block accumulators
// a.jacc[grid].
cudaError_t launch_adj_jtne(const ModelConst<double>& K, const AdjArgs& a, int grid,
                            cudaStream_t s);

} // namespace lbk
