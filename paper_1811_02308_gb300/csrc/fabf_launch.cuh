// Kernel launch helpers, instantiated once per precision in
// fabf_inst_fp64.cu, fabf_inst_fp64fit.cu, fabf_inst_cfp32.cu and
// fabf_inst_c32.cu, plus the centred form's 3-CTA build in fabf_inst_c32w.cu
// (separate translation units so that nvcc compiles them in parallel).
#pragma once

#include <cuda_runtime.h>

#include "fabf_internal.h"
#include "fabf_kernels.cuh"

namespace fabf {

constexpr int kMaxDynSmem = 110 * 1024;   // >= fused_smem_bytes for every (w <= 40, N <= 6, TH <= 64)

template <int N, int PREC, int MINB>
cudaError_t launch_fused_build(const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    const cudaError_t e = set_smem_limit_once<fabf_fused_kernel<N, PREC, MINB>>(kMaxDynSmem);
    if (e != cudaSuccess) return e;
    fabf_fused_kernel<N, PREC, MINB><<<grid, kThreads, smem, s>>>(tm, p);
    return cudaGetLastError();
}

template <int N, int PREC>
cudaError_t launch_fused_one(const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    if constexpr (PREC == kPrecC32) {
        // the 3-CTA build where only 3 CTAs are resident (resident_ctas)
        if (resident_ctas(PREC, N, smem) <= 3) return launch_fused_c32_wide(N, tm, p, grid, smem, s);
    }
    return launch_fused_build<N, PREC, MinBlocks<PREC>::value>(tm, p, grid, smem, s);
}

template <int PREC>
cudaError_t launch_fused_impl(int N, const CUtensorMap& tm, const FusedParams& p, dim3 grid, size_t smem,
                              cudaStream_t s)
{
    switch (N) {
    case 0: return launch_fused_one<0, PREC>(tm, p, grid, smem, s);
    case 1: return launch_fused_one<1, PREC>(tm, p, grid, smem, s);
    case 2: return launch_fused_one<2, PREC>(tm, p, grid, smem, s);
    case 3: return launch_fused_one<3, PREC>(tm, p, grid, smem, s);
    case 4: return launch_fused_one<4, PREC>(tm, p, grid, smem, s);
    case 5: return launch_fused_one<5, PREC>(tm, p, grid, smem, s);
    case 6: return launch_fused_one<6, PREC>(tm, p, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int PREC, int MINB>
cudaError_t launch_batch_build(const BatchParams& p, int grid, size_t smem, cudaStream_t s)
{
    const cudaError_t e = set_smem_limit_once<fabf_batch_kernel<PREC, MINB>>(kMaxDynSmem);
    if (e != cudaSuccess) return e;
    fabf_batch_kernel<PREC, MINB><<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_batch_impl(const BatchParams& p, int grid, size_t smem, cudaStream_t s)
{
    if constexpr (PREC == kPrecC32) {
        // the largest tile's shared memory sizes the persistent grid; where it
        // leaves 3 CTAs per SM, the 3-CTA build (more registers, no spills)
        if (smem_resident_ctas(smem) <= 3) return launch_batch_c32_wide(p, grid, smem, s);
    }
    return launch_batch_build<PREC, MinBlocks<PREC>::value>(p, grid, smem, s);
}

}  // namespace fabf
