// Instantiation of the box-cascade tiles for precision 0 (see fabf_casc_kernels.cuh).
#include "fabf_casc_kernels.cuh"

namespace fabf {

cudaError_t launch_casc_p0(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    return launch_casc_impl<0>(N, tm, p, grid, smem, s);
}

}  // namespace fabf
