// Host-side launchers of the library's kernels.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace cl {

// one scheduled operation of the factorisation / selected inversion
template <typename T, typename R>
cudaError_t launch_op(const Plan& p, const Op& op, T* arena, const double* links, double m, double mu,
                      double* Gdiag, double* Gfwd, double* Gbwd, cudaStream_t st);

// batched complex GEMM over the descriptors of one OP_GEMM
cudaError_t launch_gemm(const Plan& p, const Op& op, double2* arena, cudaStream_t st);
cudaError_t launch_gemm(const Plan& p, const Op& op, float2* arena, cudaStream_t st);

// fermion drift of every link of every replica
cudaError_t launch_drift(const Plan& p, const double* links, const double* Gfwd, const double* Gbwd, double mu,
                         double nf, double* Kf, cudaStream_t st);

}  // namespace cl
