// The 1024-thread step kernel (bonded networks), FP32.
#include "swp_internal.h"
#include "swp_wide.cuh"
namespace swp {
template cudaError_t launch_run_wide<float>(const Dev<float>&, const RunArgs&, int, cudaStream_t);
template cudaError_t run_occupancy_wide<float>(int*);
}
