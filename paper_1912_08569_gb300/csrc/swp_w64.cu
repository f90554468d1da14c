// The 1024-thread step kernel (bonded networks), FP64.
#include "swp_internal.h"
#include "swp_wide.cuh"
namespace swp {
template cudaError_t launch_run_wide<double>(const Dev<double>&, const RunArgs&, int, cudaStream_t);
template cudaError_t run_occupancy_wide<double>(int*);
}
