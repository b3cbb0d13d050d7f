// cgemm_tc.cu -- split-precision tensor-core complex GEMM for the MFT (3xTF32 / 3xBF16).
#include <cuda_runtime.h>

#include "../../include/coro.h"
#include "mft_gemm.cuh"

namespace coro {

cudaError_t launch_cgemm_tc(const GemmDesc& g, int batch, int precision, cudaStream_t stream) {
    (void)g; (void)batch; (void)precision; (void)stream;
    return cudaErrorNotSupported;
}

}  // namespace coro
