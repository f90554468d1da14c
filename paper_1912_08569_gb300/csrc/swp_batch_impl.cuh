// The batched step kernel of one block shape and its host launchers.  The
// including file defines SWP_BATCH_NS (the namespace of this shape's copy of
// the kernels), SWP_BATCH_THREADS (threads per block) and SWP_BATCH_MINB
// (blocks per SM the launch bounds ask registers for), then expands
// SWP_BATCH_DEFINE(float) and/or SWP_BATCH_DEFINE(double) inside namespace
// swp: they define launch_batch_<threads> and batch_occupancy_<threads>
// (declared in swp_internal.h) for that precision.

#define SWP_BATCHED 1
#include "swp_kernels.cuh"
#undef SWP_BATCHED

namespace swp {
namespace SWP_BATCH_NS {

template <typename Real>
static void* batch_fn(int uni, int bonds)
{
    if (bonds) return uni ? (void*)k_batch<Real, true, true> : (void*)k_batch<Real, false, true>;
    return uni ? (void*)k_batch<Real, true, false> : (void*)k_batch<Real, false, false>;
}

template <typename Real>
static cudaError_t batch_launch(const Dev<Real>* devs, const RunArgs* args, const int* item_ofs, const int4* items,
                                int uni, int bonds, int grid, cudaStream_t s)
{
    void* fn = batch_fn<Real>(uni, bonds);
    const size_t sm = Stage<Real>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    void* kargs[] = {(void*)&devs, (void*)&args, (void*)&item_ofs, (void*)&items};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), kargs, sm, s);
}

// Blocks per SM that every (uniform, bonds) variant of this shape reaches.
template <typename Real>
static cudaError_t batch_occ(int* blocks_per_sm)
{
    const int sm = (int)Stage<Real>::kBytes;
    int best = 1 << 30;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 4 && e == cudaSuccess; v++) {
        void* fn = batch_fn<Real>(v & 1, v >> 1);
        int b = 0;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kThreads, sm);
        best = b < best ? b : best;
    }
    *blocks_per_sm = best;
    return e;
}

}  // namespace SWP_BATCH_NS
}  // namespace swp

#define SWP_BATCH_CAT2(a, b) a##b
#define SWP_BATCH_CAT(a, b) SWP_BATCH_CAT2(a, b)
#define SWP_BATCH_DEFINE(R)                                                                                  \
    cudaError_t SWP_BATCH_CAT(launch_batch_, SWP_BATCH_THREADS)(const Dev<R>* devs, const RunArgs* args,    \
                                                                 const int* item_ofs, const int4* items,     \
                                                                 int uni, int bonds, int grid, cudaStream_t s) \
    {                                                                                                        \
        return SWP_BATCH_NS::batch_launch<R>(devs, args, item_ofs, items, uni, bonds, grid, s);              \
    }                                                                                                        \
    cudaError_t SWP_BATCH_CAT(batch_occupancy_, SWP_BATCH_THREADS)(Prec<R>, int* blocks_per_sm)             \
    {                                                                                                        \
        return SWP_BATCH_NS::batch_occ<R>(blocks_per_sm);                                                    \
    }
