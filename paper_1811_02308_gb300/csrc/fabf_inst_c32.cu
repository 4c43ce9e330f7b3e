// Instantiation of the tiled kernels for precision 3 (see fabf_launch.cuh).
#include "fabf_internal.h"
#include "fabf_launch.cuh"

namespace fabf {

cudaError_t launch_fused_p3(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                            cudaStream_t s)
{
    return launch_fused_impl<3>(N, tm, p, grid, smem, s);
}

cudaError_t launch_batch_p3(const BatchParams& p, int grid, size_t smem, cudaStream_t s)
{
    return launch_batch_impl<3>(p, grid, smem, s);
}

}  // namespace fabf
