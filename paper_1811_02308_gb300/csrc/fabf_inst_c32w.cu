// The centred form's fused and batch kernels compiled for 3 CTAs per SM (up to 85
// registers per thread), used where only 3 CTAs are resident anyway (see
// resident_ctas in fabf_internal.h).
#include "fabf_internal.h"
#include "fabf_launch.cuh"

namespace fabf {

cudaError_t launch_fused_c32_wide(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                                  cudaStream_t s)
{
    switch (N) {
    case 0: return launch_fused_build<0, kPrecC32, 3>(tm, p, grid, smem, s);
    case 1: return launch_fused_build<1, kPrecC32, 3>(tm, p, grid, smem, s);
    case 2: return launch_fused_build<2, kPrecC32, 3>(tm, p, grid, smem, s);
    case 3: return launch_fused_build<3, kPrecC32, 3>(tm, p, grid, smem, s);
    case 4: return launch_fused_build<4, kPrecC32, 3>(tm, p, grid, smem, s);
    case 5: return launch_fused_build<5, kPrecC32, 3>(tm, p, grid, smem, s);
    case 6: return launch_fused_build<6, kPrecC32, 3>(tm, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_c32_wide(const BatchParams& p, int grid, size_t smem, cudaStream_t s)
{
    return launch_batch_build<kPrecC32, 3>(p, grid, smem, s);
}

}  // namespace fabf
