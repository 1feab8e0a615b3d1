// corr_tc.cu -- split-precision BF16x3 correlation GEMM on the tensor cores.
#include "internal.h"

namespace fpc {

bool tc_gemm_available() { return false; }

cudaError_t launch_corr_bf16x3(const uint16_t *, const uint16_t *, long long, long long, int,
                               float *, int, float *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace fpc
