// The 1024-thread copy of the single-system step kernel (two-barrier step
// only, run by bonded networks) and its launchers; included once per
// precision (swp_w32.cu, swp_w64.cu), which instantiates them.
#pragma once

#include <algorithm>

#define SWP_BATCHED 0
#define SWP_WIDE 1
#include "swp_kernels.cuh"
#undef SWP_WIDE
#undef SWP_BATCHED

namespace swp {

template <typename Real>
static void* run_fn_wide(int uni, int bonds)
{
    if (bonds) return uni ? (void*)wide::k_run<Real, true, true> : (void*)wide::k_run<Real, false, true>;
    return uni ? (void*)wide::k_run<Real, true, false> : (void*)wide::k_run<Real, false, false>;
}

template <typename Real>
cudaError_t launch_run_wide(const Dev<Real>& d, const RunArgs& a, int grid, cudaStream_t s)
{
    void* fn = run_fn_wide<Real>(a.uni, d.has_bonds);
    const size_t sm = wide::Stage<Real>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    Dev<Real> dd = d;
    RunArgs aa = a;
    void* args[] = {(void*)&dd, (void*)&aa};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlockWide), args, sm, s);
}

// Blocks per SM that every (uniform, bonds) variant reaches.
template <typename Real>
cudaError_t run_occupancy_wide(int* blocks_per_sm)
{
    const int sm = (int)wide::Stage<Real>::kBytes;
    int best = 1 << 30;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 4 && e == cudaSuccess; v++) {
        void* fn = run_fn_wide<Real>(v & 1, v >> 1);
        int b = 0;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kBlockWide, sm);
        best = std::min(best, b);
    }
    *blocks_per_sm = best;
    return e;
}

}  // namespace swp
