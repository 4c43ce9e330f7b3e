// Instantiation of the separable-kernel tiles for precision 3 (see fabf_sep_kernels.cuh).
#include "fabf_sep_kernels.cuh"

namespace fabf {

cudaError_t launch_sep_p3(int N, const CUtensorMap& tm, const SepParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    return launch_sep_impl<3>(N, tm, p, grid, smem, s);
}

}  // namespace fabf
