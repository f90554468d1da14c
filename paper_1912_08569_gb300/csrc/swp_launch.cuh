// Host launchers of the step and exchange kernels, instantiated once per
// precision (swp_f32.cu, swp_f64.cu).
#pragma once

#include <algorithm>

#define SWP_BATCHED 0
#include "swp_kernels.cuh"
#undef SWP_BATCHED
// the batched kernel's 1024-thread shape (both precisions)
#define SWP_BATCH_NS batched1024
#define SWP_BATCH_THREADS 1024
#define SWP_BATCH_MINB 1
#include "swp_batch_impl.cuh"

namespace swp {
using single::Stage;

template <typename Real>
static void* run_fn(int uni, int bonds = 0)
{
    if (bonds) return uni ? (void*)single::k_run<Real, true, true> : (void*)single::k_run<Real, false, true>;
    return uni ? (void*)single::k_run<Real, true, false> : (void*)single::k_run<Real, false, false>;
}

template <typename Real>
size_t run_smem_bytes()
{
    // the two-barrier step's staging or the resident step's structures (one buffer)
    return std::max(Stage<Real>::kBytes, single::RStage::kBytes);
}

// Opts every variant into the dynamic shared memory it needs (once).
template <typename Real>
static cudaError_t prepare_fn(void* fn)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)run_smem_bytes<Real>());
}

template <typename Real>
cudaError_t launch_run(const Dev<Real>& d, const RunArgs& a, int grid, int block, cudaStream_t s)
{
    void* fn = run_fn<Real>(a.uni, d.has_bonds);
    cudaError_t e = prepare_fn<Real>(fn);
    if (e != cudaSuccess) return e;
    Dev<Real> dd = d;
    RunArgs aa = a;
    void* args[] = {(void*)&dd, (void*)&aa};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, run_smem_bytes<Real>(), s);
}

template <typename Real>
cudaError_t run_occupancy(int block, int* blocks_per_sm)
{
    int best = 1 << 30;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 4 && e == cudaSuccess; v++) {  // every (uniform, bonds) variant
        void* fn = run_fn<Real>(v & 1, v >> 1);
        int b = 0;
        e = prepare_fn<Real>(fn);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, block, run_smem_bytes<Real>());
        best = b < best ? b : best;
    }
    *blocks_per_sm = best;
    return e;
}

static inline int io_grid(int n) { return n > 0 ? (n + 255) / 256 : 1; }

template <typename Real>
cudaError_t launch_set_state(const Dev<Real>& d, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    single::k_set_state<Real><<<io_grid(d.n), 256, 0, s>>>(d);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_get_state(const Dev<Real>& d, int pc, int ac, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    single::k_get_state<Real><<<io_grid(d.n), 256, 0, s>>>(d, pc, ac);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_get_forces(const Dev<Real>& d, int pc, cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    single::k_get_forces<Real><<<io_grid(d.n), 256, 0, s>>>(d, pc);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_get_nlist(const Dev<Real>& d, int pc, int* rows, int* counts, int width,
                             cudaStream_t s)
{
    if (d.n == 0) return cudaSuccess;
    single::k_get_nlist<Real><<<io_grid(d.n), 256, 0, s>>>(d, pc, rows, counts, width);
    return cudaGetLastError();
}

// Parameter derivatives (k_pgrad_*): S/D per slot into sd [2n], dF/dtheta
// into out [3][n][3] (user order) when out is not null, the four sums into
// total [4]; part: scratch of 4 * 512 doubles.
template <typename Real>
cudaError_t launch_param_grad(const Dev<Real>& d, int pc, double* sd, double* part, const double* theta,
                              double* out, double* total, double* dU, cudaStream_t s)
{
    // kPgLanes threads per particle; at most 512 blocks (the partials scratch)
    const int blocks = std::max(1, std::min(512, (d.n * single::kPgLanes + 255) / 256));
    single::k_pgrad_sums<Real><<<blocks, 256, 0, s>>>(d, pc, sd, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (out) {
        single::k_pgrad_forces<Real><<<blocks, 256, 0, s>>>(d, pc, sd, theta, out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    single::k_pgrad_total<<<1, 128, 0, s>>>(part, blocks, total, theta, dU);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_eval_prep(const Dev<Real>& d, int ti, int tj, const double* theta, double c_rmin, double c_rb,
                             double rbond, const int* type, cudaStream_t s)
{
    single::k_eval_prep<Real><<<io_grid(d.n), 256, 0, s>>>(d, ti, tj, theta, c_rmin, c_rb, rbond, type);
    return cudaGetLastError();
}

#define SWP_INSTANTIATE(R)                                                                       \
    template cudaError_t launch_run<R>(const Dev<R>&, const RunArgs&, int, int, cudaStream_t);   \
    template cudaError_t run_occupancy<R>(int, int*);                                            \
    template cudaError_t launch_set_state<R>(const Dev<R>&, cudaStream_t);                       \
    template cudaError_t launch_get_state<R>(const Dev<R>&, int, int, cudaStream_t);             \
    template cudaError_t launch_get_forces<R>(const Dev<R>&, int, cudaStream_t);                 \
    template cudaError_t launch_get_nlist<R>(const Dev<R>&, int, int*, int*, int, cudaStream_t); \
    SWP_BATCH_DEFINE(R)                                                                          \
    template cudaError_t launch_param_grad<R>(const Dev<R>&, int, double*, double*, const double*, double*, \
                                              double*, double*, cudaStream_t);                            \
    template cudaError_t launch_eval_prep<R>(const Dev<R>&, int, int, const double*, double, double, double, \
                                             const int*, cudaStream_t);                                  \
    template size_t run_smem_bytes<R>();

}  // namespace swp
