// mft_gemm.cuh -- batched complex GEMM descriptors for the MFT.
#pragma once
#include <cuda_runtime.h>

namespace coro {

// C[b][m][n] = scale_b * sum_k opA[b][m][k] opB[b][k][n], all row-major complex64.
// opA[m][k] = a_trans ? A[k*lda + m] : A[m*lda + k]; opB likewise with b_trans.
// scale_b = scale_per_item ? scale_per_item[b] : alpha.
struct GemmDesc {
    int M, N, K;
    const float2* A; long long sA; int lda; bool a_trans;
    const float2* B; long long sB; int ldb; bool b_trans;
    float2* C; long long sC; int ldc;
    float alpha;
    const float* scale_per_item;
};

// precision: CORO_MFT_FP32 (CUDA cores) or the split tensor-core modes.
cudaError_t launch_cgemm(const GemmDesc& g, int batch, int precision, cudaStream_t stream);

// The same contraction in complex128 with FP64 arithmetic (CORO_MFT_FP64).
struct ZGemmDesc {
    int M, N, K;
    const double2* A; long long sA; int lda; bool a_trans;
    const double2* B; long long sB; int ldb; bool b_trans;
    double2* C; long long sC; int ldc;
    double alpha;
    const double* scale_per_item;
};
cudaError_t launch_zgemm(const ZGemmDesc& g, int batch, cudaStream_t stream);

}  // namespace coro
