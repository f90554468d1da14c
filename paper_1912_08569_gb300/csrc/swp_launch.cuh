// Host launchers of the step and exchange kernels, instantiated once per
// precision (swp_f32.cu, swp_f64.cu).
#pragma once

#include "swp_kernels.cuh"

namespace swp {

template <typename Real>
static void* run_fn(int lanes)
{
    switch (lanes) {
    case 1: return (void*)k_run<Real, 1>;
    case 2: return (void*)k_run<Real, 2>;
    case 4: return (void*)k_run<Real, 4>;
    case 8: return (void*)k_run<Real, 8>;
    case 16: return (void*)k_run<Real, 16>;
    case 32: return (void*)k_run<Real, 32>;
    default: return nullptr;
    }
}

template <typename Real>
cudaError_t launch_run(const Dev<Real>& d, const RunArgs& a, int grid, int block, int lanes,
                       cudaStream_t s)
{
    void* fn = run_fn<Real>(lanes);
    if (!fn) return cudaErrorInvalidValue;
    Dev<Real> dd = d;
    RunArgs aa = a;
    void* args[] = {(void*)&dd, (void*)&aa};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, s);
}

template <typename Real>
cudaError_t run_occupancy(int block, int lanes, int* blocks_per_sm)
{
    void* fn = run_fn<Real>(lanes);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, 0);
}

static inline int io_grid(int n) { return n > 0 ? (n + 255) / 256 : 1; }

template <typename Real>
cudaError_t launch_set_state(const Dev<Real>& d, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_set_state<Real><<<io_grid(d.n), 256, 0, s>>>(d);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_get_state(const Dev<Real>& d, int pc, int ac, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_get_state<Real><<<io_grid(d.n), 256, 0, s>>>(d, pc, ac);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_get_forces(const Dev<Real>& d, int pc, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_get_forces<Real><<<io_grid(d.n), 256, 0, s>>>(d, pc);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_get_nlist(const Dev<Real>& d, int pc, int* rows, int* counts, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    k_get_nlist<Real><<<io_grid(d.n), 256, 0, s>>>(d, pc, rows, counts);
    return cudaGetLastError();
}

#define SWP_INSTANTIATE(R)                                                                       \
    template cudaError_t launch_run<R>(const Dev<R>&, const RunArgs&, int, int, int, cudaStream_t); \
    template cudaError_t run_occupancy<R>(int, int, int*);                                       \
    template cudaError_t launch_set_state<R>(const Dev<R>&, cudaStream_t);                       \
    template cudaError_t launch_get_state<R>(const Dev<R>&, int, int, cudaStream_t);             \
    template cudaError_t launch_get_forces<R>(const Dev<R>&, int, cudaStream_t);                 \
    template cudaError_t launch_get_nlist<R>(const Dev<R>&, int, int*, int*, cudaStream_t);

}  // namespace swp
