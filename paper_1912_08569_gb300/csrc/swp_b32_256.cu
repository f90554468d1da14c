// The FP32 batched step kernel with 256-thread blocks (up to 255 registers per thread, no spills).
#include "swp_internal.h"
#define SWP_BATCH_NS batched256
#define SWP_BATCH_THREADS 256
#define SWP_BATCH_MINB 1
#include "swp_batch_impl.cuh"
namespace swp {
SWP_BATCH_DEFINE(float)
}
