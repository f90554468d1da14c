// FP64 instantiation of the step kernels.
#include "swp_launch.cuh"
namespace swp {
SWP_INSTANTIATE(double)
}
